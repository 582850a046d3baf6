/*
 * dmr.h -- C-ABI of the GB300 (sm_103a) evaluator for multi-objective dual
 * simplex-mesh deformable 3-D image registration (Andreadis, Bosman,
 * Alderliesten, arXiv 2202.11001).
 *
 * One problem = a source and a target image, two tetrahedral meshes with the
 * same topology (one per image, Sec. 2.1 "dual-dynamic grid"), optional
 * guidance point pairs (Sec. 2.3.3), and a population of candidate mesh
 * pairs.  For every candidate the library computes four minimised values,
 * in this order (FP64):
 *
 *   obj[0] f_sim  forward + backward squared intensity difference of
 *                 corresponding voxels with the black-vs-grey rule, over the
 *                 total voxel count of both images (Sec. 2.3.1)
 *   obj[1] f_def  deformation magnitude: Hooke springs on 6 edges + 4 spokes
 *                 per tetrahedron over 10*N_tet (Sec. 2.3.2, DMR_SPRING), or
 *                 linear-elastic energy from the deformation gradient with
 *                 Lame lambda, mu over the total rest volume (DMR_LINEAR)
 *   obj[2] f_guid symmetric squared distance (mm^2) of guidance pairs carried
 *                 through their containing tetrahedra, over 2*n_guide
 *                 (Sec. 2.3.3)
 *   obj[3] c_fold constraint count: inverted tetrahedra of either mesh,
 *                 border points that left their border plane (counted once
 *                 per incident tetrahedron), unlocated guidance points
 *                 (Sec. 2.3.4); the candidate is feasible iff it is 0
 *
 * Conventions
 *  - Images are [nz][ny][nx], x fastest; voxel (i,j,k) has its centre at
 *    (i,j,k) in voxel units.  Mesh point (a,b,c) rests at
 *    -0.5 + a*n/(m-1) per axis, so border points lie on the outer voxel
 *    faces; border coordinates must stay exactly there.
 *  - Mesh point id = a + m_x*(b + m_y*c).  Candidate coordinates are FP64,
 *    [C][2][3][P]: (candidate, mesh 0 = source / 1 = target, axis x/y/z,
 *    point), in voxel units of that mesh's image.
 *  - Pointers marked "host or device" may point to either; the library
 *    asks the CUDA runtime which one it is.  Every input is copied or read
 *    during the call; the caller keeps ownership of every buffer.
 *  - Work is enqueued on the problem's stream.  A call that writes to host
 *    memory synchronises that stream before it returns; a call whose outputs
 *    are all device pointers returns without waiting.
 *  - Every call returns DMR_OK or a negative status; no exception crosses
 *    the ABI.  dmr_last_error() gives the calling thread's last message.
 */
#ifndef DMR_H
#define DMR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dmr_problem dmr_problem;
typedef struct dmr_plan dmr_plan;
typedef struct dmr_batch dmr_batch;

enum {
  DMR_OK = 0,
  DMR_EINVAL = -1,   /* bad argument or size */
  DMR_ENOMEM = -2,   /* device or host allocation failed */
  DMR_ECUDA = -3,    /* a CUDA runtime call failed */
  DMR_ETIMEOUT = -4, /* a bounded device wait gave up: returned by the dmr_mlp_*
                        calls when a tensor-core completion wait runs out */
  DMR_ESTATE = -5    /* call out of order (e.g. commit before eval_partial) */
};

enum { DMR_F32 = 0, DMR_BF16 = 1, DMR_F16 = 2 };
enum { DMR_SPRING = 0, DMR_LINEAR = 1 };

typedef struct {
  const void* img[2];    /* source, target image; host or device */
  int img_dtype;         /* element type of img[]: DMR_F32 | DMR_BF16 | DMR_F16 */
  int dims[2][3];        /* (nx, ny, nz) of each image, each >= 1 */
  double spacing[2][3];  /* mm per voxel of each image, > 0 */
  int storage_dtype;     /* on-device image type: DMR_F32 | DMR_BF16 | DMR_F16 */
  int mesh_pts[3];       /* mesh points per axis (both meshes), each >= 2 */
  const double* guide;   /* [n_guide][2][3] host: source point, target point
                            (voxel units of their images); NULL if n_guide=0 */
  int n_guide;
  int black_rule;        /* 1: a black/grey voxel pair costs 1 (Sec. 2.3.1) */
  int deform_model;      /* DMR_SPRING (paper) | DMR_LINEAR */
  double lambda, mu;     /* Lame parameters of DMR_LINEAR */
  int max_candidates;    /* population capacity, >= 1 */
  void* stream;          /* cudaStream_t to enqueue on; NULL = default stream */
  const int* guide_set;  /* [n_guide] host: guidance set of each pair, or NULL.
                            Set form (Sec. 2.3.3): a source point's term is the
                            smallest squared distance from its mapped position
                            to the target points of its set, and vice versa;
                            NULL = every pair its own set (point pairs). */
} dmr_problem_desc;

/* Create a problem: uploads and converts both images, builds the mirrored
 * 6-tets-per-cube topology (Sec. 2.1, Fig. 1A/B) and the point -> tet
 * dependency table (Sec. 2.2).  *out receives a handle the caller frees
 * with dmr_problem_destroy.  DMR_EINVAL on bad sizes or types. */
int dmr_problem_create(const dmr_problem_desc* desc, dmr_problem** out);
int dmr_problem_destroy(dmr_problem* p);
int dmr_set_stream(dmr_problem* p, void* stream);
/* n_points = m_x*m_y*m_z, n_tets = 6*(m_x-1)*(m_y-1)*(m_z-1). */
int dmr_problem_info(const dmr_problem* p, int* n_points, int* n_tets);
/* Topology copy-out for inspection: tets [N_tet][4] point ids. */
int dmr_tets_out(const dmr_problem* p, int* tets);

/* Register the family of subsets (FOS) of mesh points that partial
 * evaluations move together (Sec. 2.2): group g holds the point ids
 * group_pts[group_ptr[g] .. group_ptr[g+1]) (host arrays, ids distinct
 * within a group).  The library derives each group's touched tetrahedra
 * (union of the points' stars) and colours the groups into waves whose
 * touched sets are pairwise disjoint.  Replaces any earlier FOS. */
int dmr_set_fos(dmr_problem* p, int n_groups, const int* group_ptr, const int* group_pts);
/* max_group: largest group size (the G of trial coordinate arrays);
 * max_touched: largest touched-tet count; n_waves: number of waves. */
int dmr_fos_info(const dmr_problem* p, int* max_group, int* max_touched, int* n_waves);
/* wave_ptr [n_waves+1], wave_groups [n_groups] (host). */
int dmr_fos_waves(const dmr_problem* p, int* wave_ptr, int* wave_groups);

/* Full evaluation (Sec. 2.3) of n_cand candidates; coords [n_cand][2][3][P]
 * FP64 (host or device); obj_out [n_cand][4] FP64 (host or device).
 * (Re)initialises the population: candidate c gets these coordinates and
 * its per-tetrahedron and per-landmark caches.  1 <= n_cand <= capacity. */
int dmr_eval_full(dmr_problem* p, int n_cand, const double* coords, double* obj_out);

/* Partial evaluation (Sec. 2.2): trial k moves the points of FOS group
 * group_ids[k] of candidate cand_ids[k] to trial_coords[k] ([2][3][G],
 * G = max_group, the first |group| entries used) and re-evaluates only the
 * touched tetrahedra and the guidance points located in them:
 *   new = stored - sum_{touched} old + sum_{touched} new.
 * group_ids, cand_ids: [n_trials] (host or device); trial_coords:
 * [n_trials][2][3][G] FP64 (host or device); obj_out [n_trials][4].
 * The committed state is unchanged; dmr_commit applies accepted trials.
 * The library keeps the derived trial lists of the 16 most recent
 * (group_ids, cand_ids) layouts on the device, so repeating a layout (as an
 * optimiser does every generation) uploads only trial_coords.  With obj_out
 * in device memory the call returns without waiting for the device. */
int dmr_eval_partial(dmr_problem* p, int n_trials, const int* group_ids, const int* cand_ids,
                     const double* trial_coords, double* obj_out);

/* Apply the trials of the last dmr_eval_partial whose accept[k] != 0
 * ([n_trials] uint8, host or device).  Accepted trials of one candidate must
 * touch disjoint tetrahedra (their changes are then independent, Sec. 2.2);
 * otherwise nothing is applied and DMR_EINVAL is returned (checked only
 * when accept is in host memory).  DMR_ESTATE without a prior partial. */
int dmr_commit(dmr_problem* p, const uint8_t* accept);

/* Accept-if-improves (Sec. 2.2): on the device, accept trial k iff its
 * c_fold is lower than the candidate's, or equal and its (f_sim, f_def,
 * f_guid) weakly Pareto-dominates the candidate's with one strict
 * improvement; then commit.  accept_out [n_trials] (host, device or NULL).
 * Accepted trials of one candidate must touch disjoint tetrahedra, which
 * holds when the trials of the last partial evaluation come from one wave. */
int dmr_commit_improving(dmr_problem* p, uint8_t* accept_out);

/* Copy-outs of the committed state (outputs host or device). */
int dmr_objectives_out(dmr_problem* p, int n, const int* cand_ids, double* out /*[n][4]*/);
int dmr_coords_out(dmr_problem* p, int cand, double* out /*[2][3][P]*/);
/* Per-tetrahedron voxel coverage counts [N_tet][2] (forward = source
 * voxels, backward = target voxels) and terms: ssd [N_tet][2], def [N_tet],
 * fold [N_tet]; any output pointer may be NULL. */
int dmr_terms_out(dmr_problem* p, int cand, int* cov, double* ssd, double* def, int* fold);
/* Guidance cache: loc [2][n_guide] (containing tet or -1), term [2][n_guide]. */
int dmr_landmarks_out(dmr_problem* p, int cand, int* loc, double* term);
/* Trial k of the last partial evaluation: touched tets (ascending), their
 * new coverage [n][2], ssd [n][2], def [n], fold [n].  Returns the touched
 * count (>= 0) or a negative status; outputs may be NULL. */
int dmr_trial_out(dmr_problem* p, int k, int* tets, int* cov, double* ssd, double* def, int* fold);
/* Voxel-samples (one per covered voxel per direction, Sec. 2.3.1) evaluated
 * by the device since the last reset; reset != 0 zeroes both counters of
 * dmr_sample_counts after reading. */
int dmr_samples(dmr_problem* p, long long* samples, int reset);
/* Both sample counters since the last reset: *counted as dmr_samples, and
 * *executed = the samples the rasterise-and-sample kernels actually mapped
 * through the affine map and sampled from the partner image.  The rest were
 * settled without sampling: a row of voxels that are 0 whose every sample
 * can reach only partner voxels that are 0 adds exactly 0 (black against
 * black, or 0 - 0), and an item whose reachable partner region is all 0
 * reads only its own voxels.  Either pointer (host) may be NULL, not both;
 * reset != 0 zeroes both after reading. */
int dmr_sample_counts(dmr_problem* p, long long* counted, long long* executed, int reset);

/* Generation plan (batched partial evaluation captured in one CUDA graph):
 * for every wave of the FOS in order, for every candidate in cand_ids:
 * propose trial = committed coordinates of the group + deltas, evaluate
 * partially, accept-if-improves, commit.  deltas: [n_groups][n_cand][2][3][G]
 * FP64 (host or device), copied into the plan.  The plan owns a CUDA graph;
 * dmr_plan_run launches it on the problem's stream. */
int dmr_plan_generation(dmr_problem* p, int n_cand, const int* cand_ids, const double* deltas,
                        dmr_plan** out);
int dmr_plan_run(dmr_plan* plan);
/* New proposal offsets for the next runs of a plan: deltas[q] for problem q
 * of the plan (one pointer for a single-problem plan), each laid out as at
 * plan creation, host or device memory.  Enqueued on the plan's stream
 * before any later dmr_plan_run; a host buffer in pinned memory must stay
 * unchanged until that run has started, pageable memory is read before the
 * call returns.  This is how an optimiser feeds a new generation's samples
 * into a captured plan. */
int dmr_plan_update(dmr_plan* plan, const double* const* deltas);

/* Batches of independent registration problems of uneven size (images,
 * meshes, populations): every kernel of a generation plan serves all of
 * them at once, one persistent launch per kernel and wave, all captured in
 * one CUDA graph.  probs: n handles (host array) on one device, one storage
 * dtype, each with a registered FOS and a population; the batch borrows
 * them (destroy the batch before its problems).  The plan runs on the first
 * problem's stream and uses its tile shape. */
int dmr_batch_create(int n, dmr_problem* const* probs, dmr_batch** out);
int dmr_batch_destroy(dmr_batch* batch);
/* Per problem q: n_cand[q] candidates cand_ids[q] and deltas[q]
 * [n_groups_q][n_cand[q]][2][3][G_q] (host or device), as in
 * dmr_plan_generation.  Wave w of the plan runs wave w of every problem. */
int dmr_batch_plan_generation(dmr_batch* batch, const int* n_cand, const int* const* cand_ids,
                              const double* const* deltas, dmr_plan** out);
int dmr_plan_destroy(dmr_plan* plan);

/* Kernel launches per dmr_plan_run (for accounting). */
int dmr_plan_launches(const dmr_plan* plan, int* launches);
/* Device time of the last completed dmr_plan_run, summed over its waves, of
 * the rasterise-and-sample kernels (CUDA events recorded inside the graph
 * around them, on the problem's stream; each recorded event costs the graph a
 * few microseconds, so only these are recorded).  *setup_ms is set to -1 (not
 * timed).  Call after that run has finished (e.g. after synchronising the
 * stream). */
int dmr_plan_kernel_ms(const dmr_plan* plan, float* setup_ms, float* raster_ms);

/* Tile shape of the rasterise-and-sample kernel: warps per CTA (4, 8, 16)
 * and voxels per warp iteration (32, 64, 128); both 0 = library default. */
int dmr_set_tile(dmr_problem* p, int warps_per_cta, int voxels_per_warp);
int dmr_get_tile(const dmr_problem* p, int* warps_per_cta, int* voxels_per_warp);
/* Autotuner: time the rasterise-and-sample kernel of every tile shape
 * (warps per CTA x voxels per warp iteration, 3 x 3) on a full evaluation of
 * the first n_cand committed candidates (n_cand <= 0: up to 16), keep the
 * fastest as the problem's tile and report it; ms_table [9] (host, may be
 * NULL) receives the times, row-major over warps {4,8,16} x voxels
 * {32,64,128}.  Needs a population (dmr_eval_full first); does not change
 * the committed state.  Plans created afterwards use the chosen tile. */
int dmr_autotune(dmr_problem* p, int n_cand, int* best_warps, int* best_vpw, float* ms_table);

/* Full evaluation of ONE candidate that allocates no memory.  The paper has
 * no counterpart; this is a service for callers that must not allocate at
 * evaluation time: optimiser loops that cannot afford the device
 * synchronisation cudaMalloc/cudaFree imply, and processes whose device
 * memory is owned by another allocator (a caching allocator or a pool that
 * holds the whole budget), where a library-side cudaMalloc would fail.
 * coords: device [2][3][P] FP64 (both meshes of the candidate); obj_out:
 * device [4] FP64, the same four values dmr_eval_full gives.  Limits:
 * N_tet <= 4608 and n_guide <= 512, else DMR_EINVAL; the problem must
 * belong to the current device, else DMR_EINVAL.  The problem's images,
 * topology and population state are only read; the scratch is one fixed
 * array of about 5.6 MB that every device holds from the library's load
 * until the process exits.  The first call on a device looks that array's
 * address up (cudaGetSymbolAddress) and should come before any stream
 * capture.  All calls share the array: calls that may overlap on the GPU
 * (other streams, other threads) race and must be serialised by the
 * caller.  Work is enqueued on the problem's stream; the call does not wait
 * for it. */
int dmr_eval_one_noalloc(dmr_problem* p, const double* coords, double* obj_out);

/* The paper's folding check (Sec. 2.3.4), as a cross-check of the signed
 * volumes that c_fold counts: per candidate and mesh, the number of points
 * of the committed coordinates that lie outside their link (the faces of
 * their star's tets that do not contain them), by the parity of the
 * crossings of a fixed ray (Moeller-Trumbore triangle test); border points
 * in their border plane against the polygon of the star's in-plane edges;
 * border-edge points between their two neighbours along the free axis.
 * cand_ids [n_cand] host or device; out [n_cand][2] host or device. */
int dmr_link_check(dmr_problem* p, int n_cand, const int* cand_ids, int* out);

/* Grid refinement for the multi-resolution scheme (Sec. 2.4): every cube
 * cell of both meshes gains a point in the middle of each edge, in the
 * middle of each face and at its centre, so m[a] points per axis become
 * 2 m[a] - 1.  A fine point on a coarse point copies it; otherwise it is the
 * mean of the 2, 4 or 8 coarse corners of the edge, face or cube it lies in
 * (summed in halves along the odd axes in z, y, x order, then scaled by
 * 1/2, 1/4 or 1/8), so border coordinates stay exactly on their planes.
 * coarse [n_cand][2][3][m0 m1 m2] and fine [n_cand][2][3][M0 M1 M2] FP64,
 * host or device memory, caller-owned; m[a] >= 2.  Runs on `stream` (a
 * cudaStream_t, 0 = the default stream) and returns after the result is in
 * `fine`.  DMR_EINVAL for bad sizes or null pointers. */
int dmr_refine(const double* coarse, int n_cand, const int* m, double* fine, void* stream);

/* Exact hypervolume (host code, no GPU): the measure of the union of the
 * boxes [p_i, ref] of n points of dimension d (1..6, minimisation), the
 * quality score of an approximation set (Sec. 1; the elitist archive of
 * Sec. 2.4).  pts [n][d] and ref [d] host; points not strictly below ref in
 * every coordinate add nothing.  *out receives the volume. */
int dmr_hypervolume(const double* pts, int n, int d, const double* ref, double* out);

/* Learned proposal (a network the paper does not have; its samples are
 * mixed into the method's own proposals, and every proposal is still scored
 * by the evaluator).  An MLP 256 -> 128 -> 128 -> 128 -> 6 with GELU (tanh form) maps features
 * of a (candidate, point) -- 5x5x5 trilinear patches of both images around
 * the source and target point, the correspondence offset and the position --
 * to the mean (3) and log-variance (3) of a Gaussian displacement of the
 * target-mesh point.  BF16 weights and activations, FP32 accumulation on the
 * tensor cores (tcgen05.mma, TMEM accumulators); FP32 master weights and Adam.
 * Parameters are FP32 [W1 (128x256), b1, W2 (128x128), b2, W3, b3,
 * W4 (16x128; rows 6..15 zero), b4 (16)], weights [out][in]. */
typedef struct dmr_mlp dmr_mlp;
int dmr_mlp_create(unsigned long long seed, void* stream, dmr_mlp** out);
int dmr_mlp_destroy(dmr_mlp* mlp);
int dmr_mlp_n_params(void);
/* Copy parameters out to `get` and/or in from `set` (host or device, FP32
 * [n_params]); either may be NULL.  Setting resets the Adam state. */
int dmr_mlp_params(dmr_mlp* mlp, float* get, const float* set);
/* Features of every (candidate, point) of coords (device [C][2][3][P]) into
 * X (device BF16 [C*P][256]). */
int dmr_mlp_features(dmr_problem* p, const double* coords, int C, void* X);
/* out (device FP32 [n][6]) = network(X) for X device BF16 [n][256], X
 * 16-byte aligned (it is read by the tensor memory accelerator; DMR_EINVAL
 * otherwise). */
int dmr_mlp_forward(dmr_mlp* mlp, const void* X, int n, float* out);
/* Gaussian negative log-likelihood of targets Y (device FP32 [n][3]) on
 * batch X (16-byte aligned, as for dmr_mlp_forward); gradient by backpropagation on the tensor cores; if lr > 0 one
 * Adam step.  loss_out (host, may be NULL) = mean loss before the step;
 * grad_out (host FP32 [n_params], may be NULL) = the gradient.  With both
 * NULL the call only enqueues the step on the network's stream and returns
 * without waiting; a tensor-core wait that gave up (DMR_ETIMEOUT) is then
 * reported by the next call that returns a loss, a gradient or parameters,
 * or runs a forward pass. */
int dmr_mlp_train_step(dmr_mlp* mlp, const void* X, const float* Y, int n, float lr, float* loss_out,
                       float* grad_out);

const char* dmr_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DMR_H */
