// Internal structures shared by the host API (dmr_api.cu) and the kernels
// (dmr_kernels.cu) of the GB300 dual simplex-mesh evaluator.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

struct dmr_problem;

namespace dmr {

// Image storage types (match DMR_F32 / DMR_BF16 / DMR_F16 of dmr.h).
enum { ST_F32 = 0, ST_BF16 = 1, ST_F16 = 2 };

// Everything a kernel needs to know about one registration problem.  Lives
// in device memory (an array of these for batched launches).
struct DevProblem {
  // images: plain [nz][ny][nx] and corner-packed cells
  // [(nz+2)][(ny+2)][(nx+2)] x 8 corners for cell origins -1..n per axis
  // (corner values pre-clamped to the image; f32 cells store each x pair as
  // value and difference), plus per-cell zero flags (bit0: some corner is 0,
  // bit1: all corners are 0, bits 2/3: the 4x4x4 block all / none 0).
  const void* plain[2];
  const void* cells[2];
  const uint8_t* cflag[2];
  // per cell: bit (dz+1)*16 + (dy+1)*4 + (dx+1) set when voxel (i+dx, j+dy,
  // k+dz) (clamped) is 0, for dx, dy, dz in -1..2
  const unsigned long long* cmask[2];
  // per image: count of nonzero voxels in [0, x) x [0, y) x [0, z), array
  // [(nz+1)][(ny+1)][(nx+1)] (NULL for images of 2^31 voxels or more)
  const int* nzsat[2];
  // per image: occupancy of 4x4x4 voxel blocks, bit (bx & 63) of word
  // (bz * BY + by) * W + (bx >> 6) set when block (bx, by, bz) holds a
  // nonzero voxel; BX = ceil(nx / 4), BY = ceil(ny / 4), W = ceil(BX / 64)
  const unsigned long long* occ[2];
  // the same bitmap dilated by one block: bit set when any of the 27 blocks
  // around (and including) the block holds a nonzero voxel
  const unsigned long long* occd[2];
  int n[2][3];
  double spd[2][3];
  float sp[2][3];
  int dtype;
  // topology
  int P, ntet;
  int m[3];
  const int4* tet;          // [ntet] point ids, positive rest orientation
  const uint32_t* fperm;    // [ntet] 4 faces x 8 bits: a|b<<2|c<<4|neg<<6
  const uint8_t* fixmask;   // [P] bit a: axis a fixed; bit 3+a: upper border
  const int* star_ptr;      // [P+1] point -> tets CSR
  const int* star;          // [4 ntet]
  const float* rest_vol;    // [ntet] source rest volume (mm^3), LINEAR model
  int black_rule, model;
  float lam, mu;
  double sim_norm, def_norm, guid_norm;
  int ng;
  const double* guide;      // [ng][2][3]
  // guidance sets (NULL: each pair its own set): set index of each pair,
  // set s holds the pairs gmem[gptr[s] .. gptr[s+1])
  const int* gsid;
  const int* gptr;
  const int* gmem;
  // population state
  int C;
  double* coords;           // [C][2][3][P]
  double* c_ssd;            // [C][ntet][2]
  int* c_cov;               // [C][ntet][2]
  double* c_def;            // [C][ntet]
  int* c_fold;              // [C][ntet]
  int* c_loc;               // [C][2][ng]
  double* c_gterm;          // [C][2][ng]
  double* sums;             // [C][4] raw sums
  unsigned long long* samples;   // voxel-samples evaluated (covered voxels of every evaluated tet)
  unsigned long long* executed;  // of those, samples the raster kernels mapped and sampled
};

// Per (trial, tet, direction) set-up produced by the geometry kernel and
// consumed by the rasterise-and-sample kernel and the landmark kernels.
// "own" = the mesh whose voxels are visited (direction 0: source, 1: target),
// "partner" = the other mesh.  Relative coordinates are taken against the
// integer origins O (own) and Op (partner).
struct __align__(16) ItemRec {
  int flags;        // bit0: rasterise (6V_own > 0); bit1: clamp-free map; bit2 / bit3: every
                    // partner voxel a sample of this item can reach is 0 / is not 0; bit4 (with
                    // bit2): the own voxels are 0 too; bit5: the FP32 map is finite and small
                    // (the rows' empty-space test may use it)
  int prob;
  int tet;
  int dir;
  int b0[4];        // clipped integer bbox, abs voxel coords (x,y,z,-)
  int b1[4];
  int O[4];         // own origin (floor of min vertex coords)
  int Op[4];        // partner origin
  unsigned cbase;   // corner-cell index offset (mod 2^32, see kernels)
  int forder;       // the faces sorted by the sign of their FP32 normal's x (2 bits each)
  int fshape;       // (faces with A.x > 0) | (faces with A.x < 0) << 4
  int pad0;
  float vr[4][4];   // own vertices relative to O (x,y,z,-)
  float fa[4][4];   // face f: inward normal A (x,y,z), offset B'
  float fm[4][4];   // face f: margin mu (box points), 1/A.x, margin growth per voxel of |p - O|,
                    // bound on the rounding error of A.x
  float G[3][4];    // map matrix rows (FP32), col 3 = k (offset)
  float gx[4];      // (1+G00, G10, G20, delta)
  float clo[4];     // clamp range of partner-relative mapped coords
  float chi[4];
  double X[4][3];   // own vertices FP64 (abs)
  double XP[4][3];  // partner vertices FP64 (abs): the exact map is rebuilt from them
};

// Kernels one launch_raster call launches (fast, full-logic).
constexpr int kRasterLaunches = 2;

// A batch of (trial, tet) pairs to evaluate.
struct Batch {
  int n_tt;
  const int* tt_trial;      // [n_tt]
  const int* tt_tet;        // [n_tt] ascending within a trial
  const uint32_t* tt_slot;  // [n_tt] 4 x 8 bit: (group slot + 1) of vertex i, 0 = unmoved; NULL = none
  int n_trials;
  const int* tr_prob;       // [n_trials] or NULL (problem 0)
  const int* tr_cand;       // [n_trials]
  const int* tr_first;      // [n_trials] first tt index
  const int* tr_ntt;        // [n_trials]
  const double* tr_coords;  // [n_trials][2][3][gmax] or NULL (full evaluation)
  int gmax;
  ItemRec* rec;             // [2 n_tt]
  double* o_ssd;            // [n_tt][2]
  int* o_cov;               // [n_tt][2]
  double* o_def;            // [n_tt]
  int* o_fold;              // [n_tt]
  unsigned* work;           // [3] raster counters: fast-kernel items taken, items handed over, handed-over items taken
  int* slow;                // [2 n_tt] items the fast raster kernel hands to the full-logic kernel
  // partial-evaluation landmark outputs
  int aff_cap;
  int* aff_n;               // [n_trials]
  int* aff_idx;             // [n_trials][aff_cap]  mesh*ng + i
  int* aff_loc;             // [n_trials][aff_cap]
  double* aff_term;         // [n_trials][aff_cap]
  double* tr_delta;         // [n_trials][4]
  double* tr_obj;           // [n_trials][4]
};

// Kernel launchers (dmr_kernels.cu).  All enqueue on `st`.
void launch_convert_image(const void* src, int src_dtype, void* dst, int dst_dtype, long n, cudaStream_t st);
void launch_build_cells(const void* plain, int dtype, const int n[3], void* cells, uint8_t* cflag,
                        unsigned long long* cmask, cudaStream_t st);
// Summed nonzero counts of an image (DevProblem::nzsat); sat holds
// (nx+1)(ny+1)(nz+1) ints.
void launch_build_nzsat(const void* plain, int dtype, const int n[3], int* sat, cudaStream_t st);
// Block occupancy bitmap (DevProblem::occ); occ holds occ_words(n) words,
// zeroed by the launch.
long occ_words(const int n[3]);
void launch_build_occ(const void* plain, int dtype, const int n[3], unsigned long long* occ, cudaStream_t st);
// occd (occ_words(n) words, zeroed by the launch) = occ dilated by one block.
void launch_dilate_occ(const unsigned long long* occ, const int n[3], unsigned long long* occd, cudaStream_t st);
void launch_setup(const DevProblem* probs, const Batch& b, cudaStream_t st);
void launch_refine(const double* coarse, int n_cand, const int m[3], double* fine, cudaStream_t st);
void launch_link_check(const DevProblem* probs, const DevProblem& hp, const int* cands, int n_cand, int* out,
                       cudaStream_t st);
void launch_gather_deltas(const double* const* raw, const int* slot_q, const long long* slot_src, const int* raw_G,
                          int n_slots, int G, double* out, cudaStream_t st);
// Raster kernels: fast pass, then the full-logic pass over the items it
// handed over.  With a side stream, `fork` is recorded on `st` before the
// fast pass and the side stream waits on it: work placed there (the guidance
// points) fills the SM slots the persistent fast pass leaves free, mostly in
// its tail and beside the full-logic pass.
void launch_raster(const DevProblem* probs, const Batch& b, int storage_dtype, int warps, int vpw, int n_sm,
                   cudaStream_t st, cudaStream_t side = nullptr, cudaEvent_t fork = nullptr);
void launch_raster_f32(const DevProblem* probs, const Batch& b, int warps, int vpw, int n_sm, cudaStream_t st,
                       cudaStream_t side, cudaEvent_t fork);
void launch_raster_bf16(const DevProblem* probs, const Batch& b, int warps, int vpw, int n_sm, cudaStream_t st,
                        cudaStream_t side, cudaEvent_t fork);
void launch_raster_f16(const DevProblem* probs, const Batch& b, int warps, int vpw, int n_sm, cudaStream_t st,
                       cudaStream_t side, cudaEvent_t fork);
void launch_locate_full(const DevProblem* probs, const DevProblem& host_pr, const Batch& b, int c0, int nc,
                        cudaStream_t st);
void launch_reduce_full(const DevProblem* probs, int c0, int nc, const Batch& b, double* obj, cudaStream_t st);
void launch_landmarks_partial(const DevProblem* probs, const Batch& b, cudaStream_t st);
void launch_reduce_partial(const DevProblem* probs, const Batch& b, cudaStream_t st);
void launch_accept(const DevProblem* probs, const Batch& b, uint8_t* accept, cudaStream_t st);
void launch_commit(const DevProblem* probs, const Batch& b, const uint8_t* accept, const int* tr_group,
                   const int* g_ptr, const int* g_pts, const int* cand_ptr, const int* cand_trials, int n_list,
                   cudaStream_t st);
// Plans: reduce + accept + per-trial commit fused, then the per-candidate sums
// (two launches instead of five).  With a side stream the sums kernel runs
// there, after `sums_ev` is recorded on `st`: beside the next wave's proposal
// and set-up, which neither read nor write what it touches.
void launch_reduce_commit(const DevProblem* probs, const Batch& b, uint8_t* accept, const int* tr_group,
                          const int* g_ptr, const int* g_pts, const int* cand_ptr, const int* cand_trials, int n_list,
                          cudaStream_t st, cudaStream_t sums_st = nullptr, cudaEvent_t sums_ev = nullptr);
void launch_propose(const DevProblem* probs, const Batch& b, const int* tr_group, const int* g_ptr, const int* g_pts,
                    const double* deltas, cudaStream_t st);

// Host helpers shared by the C-ABI translation units (dmr_api.cu).
// Record the calling thread's error message and return `code`.
int set_error(int code, const std::string& msg);
// Host copy of a problem's device descriptor plus its launch settings.
int problem_view(const ::dmr_problem* p, DevProblem* hp, int* storage, int* warps, int* n_sm, cudaStream_t* st);
// The problem's device descriptor (an array of one).
const DevProblem* problem_device(const ::dmr_problem* p);
// The CUDA device the problem was created on (-1 for a null problem).
int problem_device_id(const ::dmr_problem* p);

}  // namespace dmr
