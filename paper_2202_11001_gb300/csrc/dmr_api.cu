// Host side of the C-ABI declared in include/dmr.h: problem lifecycle,
// mesh topology (Sec. 2.1), FOS registration and wave colouring (Sec. 2.2),
// and the orchestration of full / partial evaluation, commit and the
// CUDA-graph generation plan.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <cstring>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "../../include/dmr.h"
#include "dmr_internal.cuh"

using namespace dmr;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CU(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return fail(DMR_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class T>
int dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(DMR_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return DMR_OK;
}

template <class T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

size_t dtype_size(int dt) { return dt == DMR_F32 ? 4 : 2; }

// Scratch for one batch of (trial, tet) pairs.
struct Scratch {
  int cap_tt = 0, cap_tr = 0, gmax = 0, aff_cap = 0;
  ItemRec* rec = nullptr;
  double* o_ssd = nullptr;
  int* o_cov = nullptr;
  double* o_def = nullptr;
  int* o_fold = nullptr;
  int* tt_trial = nullptr;
  int* tt_tet = nullptr;
  uint32_t* tt_slot = nullptr;
  int* tr_cand = nullptr;
  int* tr_first = nullptr;
  int* tr_ntt = nullptr;
  int* tr_group = nullptr;
  double* tr_coords = nullptr;
  int* aff_n = nullptr;
  int* aff_idx = nullptr;
  int* aff_loc = nullptr;
  double* aff_term = nullptr;
  double* tr_delta = nullptr;
  double* tr_obj = nullptr;
  uint8_t* accept = nullptr;
  int* cand_ptr = nullptr;
  int* cand_trials = nullptr;
  unsigned* work = nullptr;
  int* slow = nullptr;

  void release() {
    dfree(rec); dfree(o_ssd); dfree(o_cov); dfree(o_def); dfree(o_fold);
    dfree(tt_trial); dfree(tt_tet); dfree(tt_slot);
    dfree(tr_cand); dfree(tr_first); dfree(tr_ntt); dfree(tr_group); dfree(tr_coords);
    dfree(aff_n); dfree(aff_idx); dfree(aff_loc); dfree(aff_term);
    dfree(tr_delta); dfree(tr_obj); dfree(accept); dfree(cand_ptr); dfree(cand_trials); dfree(work);
    dfree(slow);
    cap_tt = cap_tr = 0;
  }

  int ensure(int ntt, int ntr, int gm, int acap) {
    if (ntt <= cap_tt && ntr <= cap_tr && gm <= gmax && acap <= aff_cap) return DMR_OK;
    int nt = std::max(ntt, cap_tt), nr = std::max(ntr, cap_tr), g = std::max(gm, gmax), a = std::max(acap, aff_cap);
    release();
    int rc = DMR_OK;
    if ((rc = dalloc(&rec, 2 * (size_t)nt)) || (rc = dalloc(&o_ssd, 2 * (size_t)nt)) ||
        (rc = dalloc(&o_cov, 2 * (size_t)nt)) || (rc = dalloc(&o_def, (size_t)nt)) ||
        (rc = dalloc(&o_fold, (size_t)nt)) || (rc = dalloc(&tt_trial, (size_t)nt)) ||
        (rc = dalloc(&tt_tet, (size_t)nt)) || (rc = dalloc(&tt_slot, (size_t)nt)) ||
        (rc = dalloc(&tr_cand, (size_t)nr)) || (rc = dalloc(&tr_first, (size_t)nr)) ||
        (rc = dalloc(&tr_ntt, (size_t)nr)) || (rc = dalloc(&tr_group, (size_t)nr)) ||
        (rc = dalloc(&tr_coords, (size_t)nr * 6 * std::max(g, 1))) || (rc = dalloc(&aff_n, (size_t)nr)) ||
        (rc = dalloc(&aff_idx, (size_t)nr * std::max(a, 1))) || (rc = dalloc(&aff_loc, (size_t)nr * std::max(a, 1))) ||
        (rc = dalloc(&aff_term, (size_t)nr * std::max(a, 1))) || (rc = dalloc(&tr_delta, (size_t)nr * 4)) ||
        (rc = dalloc(&tr_obj, (size_t)nr * 4)) || (rc = dalloc(&accept, (size_t)nr)) ||
        (rc = dalloc(&cand_ptr, (size_t)nr + 1)) || (rc = dalloc(&cand_trials, (size_t)nr)) ||
        (rc = dalloc(&work, 4)) || (rc = dalloc(&slow, 2 * (size_t)nt))) {
      release();
      return rc;
    }
    cap_tt = nt;
    cap_tr = nr;
    gmax = g;
    aff_cap = a;
    return DMR_OK;
  }
};

}  // namespace

namespace {
// A trial layout of dmr_eval_partial (the group and candidate of every
// trial) with its derived lists, on the host and on the device.  Optimisers
// repeat the same layouts every generation (one per wave), so the library
// keeps the most recent ones and a repeated call uploads only the trial
// coordinates.
struct Layout {
  std::vector<int> gid, cid, first, ntt, cptr, ctr;
  int tot = 0, max_cid = 0;
  bool safe = true;
  unsigned long long used = 0;
  int *tt_trial = nullptr, *tt_tet = nullptr, *tr_cand = nullptr, *tr_group = nullptr, *tr_first = nullptr,
      *tr_ntt = nullptr, *cand_ptr = nullptr, *cand_trials = nullptr;
  uint32_t* tt_slot = nullptr;
  void release() {
    dfree(tt_trial); dfree(tt_tet); dfree(tt_slot); dfree(tr_cand); dfree(tr_group); dfree(tr_first); dfree(tr_ntt);
    dfree(cand_ptr); dfree(cand_trials);
  }
};
constexpr int kLayoutCache = 16;
}  // namespace

struct dmr_problem {
  int dev = 0;
  cudaStream_t st = nullptr;
  // side stream for landmark relocation beside the raster kernels (lazy)
  cudaStream_t st2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int n_sm = 1;
  int P = 0, ntet = 0, m[3] = {0, 0, 0};
  int n[2][3];
  double sp[2][3];
  int storage = DMR_F32;
  int black_rule = 1, model = DMR_SPRING;
  double lam = 1, mu = 1;
  int ng = 0;
  int cap = 0, C = 0;
  std::vector<int> tets;
  std::vector<uint32_t> fperm;
  std::vector<uint8_t> fixmask;
  std::vector<int> star_ptr, star;
  std::vector<double> guide;
  // device state
  void* plain[2] = {nullptr, nullptr};
  void* cells[2] = {nullptr, nullptr};
  uint8_t* cflag[2] = {nullptr, nullptr};
  unsigned long long* cmask[2] = {nullptr, nullptr};
  int* nzsat[2] = {nullptr, nullptr};
  unsigned long long* occ[2] = {nullptr, nullptr};
  unsigned long long* occd[2] = {nullptr, nullptr};
  int4* d_tet = nullptr;
  uint32_t* d_fperm = nullptr;
  uint8_t* d_fix = nullptr;
  int* d_star_ptr = nullptr;
  int* d_star = nullptr;
  float* d_restvol = nullptr;
  double* d_guide = nullptr;
  std::vector<int> gs_id, gs_ptr, gs_mem;  // guidance sets (empty: one set per pair)
  int* d_gs_id = nullptr;
  int* d_gs_ptr = nullptr;
  int* d_gs_mem = nullptr;
  double* d_coords = nullptr;
  double* d_ssd = nullptr;
  int* d_cov = nullptr;
  double* d_def = nullptr;
  int* d_fold = nullptr;
  int* d_loc = nullptr;
  double* d_gterm = nullptr;
  double* d_sums = nullptr;
  unsigned long long* d_samples = nullptr;
  DevProblem hp;
  DevProblem* d_prob = nullptr;
  double* d_obj = nullptr;  // [cap][4] staging for objective outputs
  // FOS
  int n_groups = 0, gmax = 0, max_touched = 0;
  std::vector<int> g_ptr, g_pts, g_tptr, g_tets, wave_ptr, wave_groups;
  std::vector<uint32_t> g_slot;
  int* d_gptr = nullptr;
  int* d_gpts = nullptr;
  // scratch and last partial evaluation
  Scratch sc;
  bool have_partial = false, partial_safe = false;
  std::vector<Layout*> layouts;  // recent eval_partial layouts
  unsigned long long layout_clock = 0;
  Layout* cur = nullptr;         // layout of the last eval_partial
  int last_ntr = 0, last_ntt = 0;
  std::vector<int> last_cand, last_group, last_first, last_ntt_v;
  int last_nlist = 0;
  int warps = 8, vpw = 32;
};

struct dmr_plan {
  dmr_problem* p = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int launches = 0;
  // per wave: events before set-up, before and after the raster kernel
  std::vector<cudaEvent_t> ev;
  // all waves' arrays (device), owned by the plan
  int* tt_trial = nullptr;
  int* tt_tet = nullptr;
  uint32_t* tt_slot = nullptr;
  int* tr_cand = nullptr;
  int* tr_first = nullptr;
  int* tr_ntt = nullptr;
  int* tr_group = nullptr;
  int* tr_prob = nullptr;
  double* deltas = nullptr;
  int* cand_ptr = nullptr;
  int* cand_trials = nullptr;
  Scratch sc;  // per-wave scratch (largest wave)
  // dmr_plan_update: per plan trial its problem and offset in that problem's
  // [n_groups][n_cand][2][3][G_q] deltas; staging copies of those arrays
  int G = 1;
  std::vector<size_t> raw_count;  // per problem
  std::vector<int> raw_G;
  int* slot_q = nullptr;
  long long* slot_src = nullptr;
  std::vector<double*> raw;       // device staging per problem
  const double** d_raw = nullptr; // device array of the source pointers
  int* d_rawG = nullptr;          // device array of G_q
  int n_slots = 0;
};

// ------------------------------------------------------------ topology
namespace {

const int kAxisOrder[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

// Mirrored 6-tets-per-cube lattice (Sec. 2.1, Fig. 1A/B): each cube is cut
// along the diagonal from its even-index corner to its odd-index corner; the
// 6 tets follow the 6 axis orders along it; orientation made positive.
void build_topology(dmr_problem* p) {
  const int mx = p->m[0], my = p->m[1], mz = p->m[2];
  p->P = mx * my * mz;
  p->ntet = 6 * (mx - 1) * (my - 1) * (mz - 1);
  p->tets.assign(4 * (size_t)p->ntet, 0);
  p->fperm.assign(p->ntet, 0u);
  auto pid = [&](int a, int b, int c) { return a + mx * (b + my * c); };
  int t = 0;
  for (int cz = 0; cz < mz - 1; ++cz)
    for (int cy = 0; cy < my - 1; ++cy)
      for (int cx = 0; cx < mx - 1; ++cx) {
        int cube[3] = {cx, cy, cz}, s0[3], dir[3];
        for (int k = 0; k < 3; ++k) {
          s0[k] = cube[k] + (cube[k] & 1);
          dir[k] = (cube[k] & 1) ? -1 : 1;
        }
        for (int q = 0; q < 6; ++q, ++t) {
          int v[4][3];
          for (int k = 0; k < 3; ++k) v[0][k] = s0[k];
          for (int s = 0; s < 3; ++s) {
            for (int k = 0; k < 3; ++k) v[s + 1][k] = v[s][k];
            v[s + 1][kAxisOrder[q][s]] += dir[kAxisOrder[q][s]];
          }
          long a[3][3];
          for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) a[i][k] = v[i + 1][k] - v[0][k];
          long det = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
                     a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
          int id[4];
          for (int i = 0; i < 4; ++i) id[i] = pid(v[i][0], v[i][1], v[i][2]);
          if (det < 0) std::swap(id[1], id[2]);
          for (int i = 0; i < 4; ++i) p->tets[4 * (size_t)t + i] = id[i];
          // faces: canonical vertex order and inward sign
          uint32_t packed = 0;
          for (int f = 0; f < 4; ++f) {
            int l[3], k = 0;
            for (int i = 0; i < 4; ++i)
              if (i != f) l[k++] = i;
            std::sort(l, l + 3, [&](int x, int y) { return id[x] < id[y]; });
            int perm[4] = {l[0], l[1], l[2], f}, inv = 0;
            for (int i = 0; i < 4; ++i)
              for (int j = i + 1; j < 4; ++j)
                if (perm[i] > perm[j]) ++inv;
            uint32_t byte = (uint32_t)l[0] | ((uint32_t)l[1] << 2) | ((uint32_t)l[2] << 4) | ((uint32_t)(inv & 1) << 6);
            packed |= byte << (8 * f);
          }
          p->fperm[t] = packed;
        }
      }
  p->star_ptr.assign(p->P + 1, 0);
  for (int tt = 0; tt < p->ntet; ++tt)
    for (int i = 0; i < 4; ++i) p->star_ptr[p->tets[4 * (size_t)tt + i] + 1]++;
  for (int v = 0; v < p->P; ++v) p->star_ptr[v + 1] += p->star_ptr[v];
  p->star.assign(4 * (size_t)p->ntet, 0);
  std::vector<int> fill(p->star_ptr.begin(), p->star_ptr.end() - 1);
  for (int tt = 0; tt < p->ntet; ++tt)
    for (int i = 0; i < 4; ++i) p->star[fill[p->tets[4 * (size_t)tt + i]]++] = tt;
  p->fixmask.assign(p->P, 0);
  for (int c = 0; c < mz; ++c)
    for (int b = 0; b < my; ++b)
      for (int a = 0; a < mx; ++a) {
        int idx[3] = {a, b, c};
        uint8_t fm = 0;
        for (int ax = 0; ax < 3; ++ax) {
          if (idx[ax] == 0) fm |= (uint8_t)(1 << ax);
          if (idx[ax] == p->m[ax] - 1) fm |= (uint8_t)((1 << ax) | (1 << (3 + ax)));
        }
        p->fixmask[pid(a, b, c)] = fm;
      }
}

void clear_layouts(dmr_problem* p) {
  for (Layout* L : p->layouts) {
    L->release();
    delete L;
  }
  p->layouts.clear();
  p->cur = nullptr;
}

void release_problem(dmr_problem* p) {
  clear_layouts(p);
  for (int k = 0; k < 2; ++k) {
    dfree(p->plain[k]);
    dfree(p->cells[k]);
    dfree(p->cflag[k]);
    dfree(p->cmask[k]);
    dfree(p->nzsat[k]);
    dfree(p->occ[k]);
    dfree(p->occd[k]);
  }
  dfree(p->d_tet); dfree(p->d_fperm); dfree(p->d_fix); dfree(p->d_restvol); dfree(p->d_guide);
  dfree(p->d_star_ptr); dfree(p->d_star);
  dfree(p->d_gs_id); dfree(p->d_gs_ptr); dfree(p->d_gs_mem);
  dfree(p->d_coords); dfree(p->d_ssd); dfree(p->d_cov); dfree(p->d_def); dfree(p->d_fold);
  dfree(p->d_loc); dfree(p->d_gterm); dfree(p->d_sums); dfree(p->d_samples); dfree(p->d_prob); dfree(p->d_obj);
  dfree(p->d_gptr); dfree(p->d_gpts);
  p->sc.release();
}

int upload_prob(dmr_problem* p) {
  CU(cudaMemcpyAsync(p->d_prob, &p->hp, sizeof(DevProblem), cudaMemcpyHostToDevice, p->st));
  return DMR_OK;
}

int copy_out(void* dst, const void* src, size_t bytes, cudaStream_t st, bool& host_dst) {
  host_dst = !is_device_ptr(dst);
  CU(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
  return DMR_OK;
}

}  // namespace

namespace dmr {

int set_error(int code, const std::string& msg) { return fail(code, msg); }

int problem_view(const ::dmr_problem* p, DevProblem* hp, int* storage, int* warps, int* n_sm, cudaStream_t* st) {
  if (!p) return fail(DMR_EINVAL, "null problem");
  *hp = p->hp;
  *storage = p->storage;
  *warps = p->warps;
  *n_sm = p->n_sm;
  *st = p->st;
  return DMR_OK;
}

const DevProblem* problem_device(const ::dmr_problem* p) { return p ? p->d_prob : nullptr; }

int problem_device_id(const ::dmr_problem* p) { return p ? p->dev : -1; }

}  // namespace dmr

extern "C" {

const char* dmr_last_error(void) { return g_err.c_str(); }

int dmr_problem_create(const dmr_problem_desc* d, dmr_problem** out) {
  if (!d || !out) return fail(DMR_EINVAL, "null argument");
  *out = nullptr;
  for (int k = 0; k < 2; ++k) {
    if (!d->img[k]) return fail(DMR_EINVAL, "image pointer is null");
    for (int a = 0; a < 3; ++a) {
      if (d->dims[k][a] < 1 || d->dims[k][a] > (1 << 20)) return fail(DMR_EINVAL, "image dims out of range");
      if (!(d->spacing[k][a] > 0) || !std::isfinite(d->spacing[k][a])) return fail(DMR_EINVAL, "spacing must be > 0");
    }
    if ((long)(d->dims[k][0] + 2) * (d->dims[k][1] + 2) * (d->dims[k][2] + 2) > (1L << 31))
      return fail(DMR_EINVAL, "image too large");
  }
  for (int a = 0; a < 3; ++a)
    if (d->mesh_pts[a] < 2 || d->mesh_pts[a] > 4096) return fail(DMR_EINVAL, "mesh_pts must be >= 2");
  if ((long)d->mesh_pts[0] * d->mesh_pts[1] * d->mesh_pts[2] > (1L << 24)) return fail(DMR_EINVAL, "mesh too large");
  if (d->img_dtype < 0 || d->img_dtype > 2 || d->storage_dtype < 0 || d->storage_dtype > 2)
    return fail(DMR_EINVAL, "bad dtype");
  if (d->deform_model != DMR_SPRING && d->deform_model != DMR_LINEAR) return fail(DMR_EINVAL, "bad deform_model");
  if (d->n_guide < 0 || (d->n_guide > 0 && !d->guide)) return fail(DMR_EINVAL, "bad guidance arguments");
  if (d->max_candidates < 1) return fail(DMR_EINVAL, "max_candidates must be >= 1");
  dmr_problem* p = new (std::nothrow) dmr_problem();
  if (!p) return fail(DMR_ENOMEM, "host allocation failed");
  int rc = DMR_OK;
  cudaGetDevice(&p->dev);
  cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, p->dev);
  p->st = (cudaStream_t)d->stream;
  for (int k = 0; k < 2; ++k)
    for (int a = 0; a < 3; ++a) {
      p->n[k][a] = d->dims[k][a];
      p->sp[k][a] = d->spacing[k][a];
    }
  for (int a = 0; a < 3; ++a) p->m[a] = d->mesh_pts[a];
  p->storage = d->storage_dtype;
  p->black_rule = d->black_rule;
  p->model = d->deform_model;
  p->lam = d->lambda;
  p->mu = d->mu;
  p->ng = d->n_guide;
  p->cap = d->max_candidates;
  p->guide.assign(d->guide ? d->guide : (const double*)nullptr, d->guide ? d->guide + 6 * (size_t)p->ng : nullptr);
  for (double g : p->guide)
    if (!std::isfinite(g)) {
      delete p;
      return fail(DMR_EINVAL, "non-finite guidance coordinate");
    }
  if (d->guide_set && p->ng > 0) {
    // compact set ids in order of first appearance; members in pair order
    std::vector<int> ids(d->guide_set, d->guide_set + p->ng), uniq;
    p->gs_id.resize(p->ng);
    for (int i = 0; i < p->ng; ++i) {
      auto it = std::find(uniq.begin(), uniq.end(), ids[i]);
      p->gs_id[i] = (int)(it - uniq.begin());
      if (it == uniq.end()) uniq.push_back(ids[i]);
    }
    p->gs_ptr.assign(uniq.size() + 1, 0);
    for (int i = 0; i < p->ng; ++i) ++p->gs_ptr[p->gs_id[i] + 1];
    for (size_t k = 0; k < uniq.size(); ++k) p->gs_ptr[k + 1] += p->gs_ptr[k];
    p->gs_mem.resize(p->ng);
    std::vector<int> fill(p->gs_ptr.begin(), p->gs_ptr.end() - 1);
    for (int i = 0; i < p->ng; ++i) p->gs_mem[fill[p->gs_id[i]]++] = i;
  }
  build_topology(p);
  // images: input -> storage, plain + corner-packed cells
  for (int k = 0; k < 2; ++k) {
    long nv = (long)p->n[k][0] * p->n[k][1] * p->n[k][2];
    long nc = (long)(p->n[k][0] + 2) * (p->n[k][1] + 2) * (p->n[k][2] + 2);
    if ((rc = dalloc((char**)&p->plain[k], nv * dtype_size(p->storage)))) goto fail_;
    if ((rc = dalloc((char**)&p->cells[k], nc * 8 * dtype_size(p->storage)))) goto fail_;
    if ((rc = dalloc(&p->cflag[k], nc))) goto fail_;
    if ((rc = dalloc(&p->cmask[k], nc))) goto fail_;
    void* src = (void*)d->img[k];
    void* tmp = nullptr;
    if (!is_device_ptr(src)) {
      if ((rc = dalloc((char**)&tmp, nv * dtype_size(d->img_dtype)))) goto fail_;
      cudaMemcpyAsync(tmp, src, nv * dtype_size(d->img_dtype), cudaMemcpyHostToDevice, p->st);
      src = tmp;
    }
    launch_convert_image(src, d->img_dtype, p->plain[k], p->storage, nv, p->st);
    launch_build_cells(p->plain[k], p->storage, p->n[k], p->cells[k], p->cflag[k], p->cmask[k], p->st);
    {
      // nonzero counts fit an int below 2^31 voxels; larger images go without
      const long ns = (long)(p->n[k][0] + 1) * (p->n[k][1] + 1) * (p->n[k][2] + 1);
      if (nv < (1L << 31)) {
        if ((rc = dalloc(&p->nzsat[k], ns)) || (rc = dalloc(&p->occ[k], occ_words(p->n[k]))) ||
            (rc = dalloc(&p->occd[k], occ_words(p->n[k]))))
          goto fail_;
        launch_build_nzsat(p->plain[k], p->storage, p->n[k], p->nzsat[k], p->st);
        launch_build_occ(p->plain[k], p->storage, p->n[k], p->occ[k], p->st);
        launch_dilate_occ(p->occ[k], p->n[k], p->occd[k], p->st);
      }
    }
    if (tmp) {
      cudaStreamSynchronize(p->st);
      cudaFree(tmp);
    }
    if (cudaGetLastError() != cudaSuccess) {
      rc = fail(DMR_ECUDA, "image preparation failed");
      goto fail_;
    }
  }
  {
    // topology + rest volumes
    std::vector<int4> t4(p->ntet);
    for (int t = 0; t < p->ntet; ++t)
      t4[t] = make_int4(p->tets[4 * t], p->tets[4 * t + 1], p->tets[4 * t + 2], p->tets[4 * t + 3]);
    std::vector<float> rv(p->ntet);
    for (int t = 0; t < p->ntet; ++t) {
      double X[4][3];
      for (int i = 0; i < 4; ++i) {
        int v = p->tets[4 * t + i];
        int idx[3] = {v % p->m[0], (v / p->m[0]) % p->m[1], v / (p->m[0] * p->m[1])};
        for (int a = 0; a < 3; ++a)
          X[i][a] = ((double)idx[a] * (double)p->n[0][a] / (double)(p->m[a] - 1) - 0.5) * p->sp[0][a];
      }
      double e[3][3];
      for (int i = 0; i < 3; ++i)
        for (int a = 0; a < 3; ++a) e[i][a] = X[i + 1][a] - X[0][a];
      double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) - e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                   e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
      rv[t] = (float)(std::fabs(det) / 6.0);
    }
    double rvs = 0;
    for (int t = 0; t < p->ntet; ++t) {
      double X[4][3];
      for (int i = 0; i < 4; ++i) {
        int v = p->tets[4 * t + i];
        int idx[3] = {v % p->m[0], (v / p->m[0]) % p->m[1], v / (p->m[0] * p->m[1])};
        for (int a = 0; a < 3; ++a)
          X[i][a] = ((double)idx[a] * (double)p->n[0][a] / (double)(p->m[a] - 1) - 0.5) * p->sp[0][a];
      }
      double e[3][3];
      for (int i = 0; i < 3; ++i)
        for (int a = 0; a < 3; ++a) e[i][a] = X[i + 1][a] - X[0][a];
      double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) - e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                   e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
      rvs += std::fabs(det) / 6.0;
    }
    size_t C = p->cap;
    if ((rc = dalloc(&p->d_star_ptr, p->star_ptr.size())) || (rc = dalloc(&p->d_star, p->star.size())))
      goto fail_;
    cudaMemcpyAsync(p->d_star_ptr, p->star_ptr.data(), sizeof(int) * p->star_ptr.size(), cudaMemcpyHostToDevice, p->st);
    cudaMemcpyAsync(p->d_star, p->star.data(), sizeof(int) * p->star.size(), cudaMemcpyHostToDevice, p->st);
    if ((rc = dalloc(&p->d_tet, p->ntet)) || (rc = dalloc(&p->d_fperm, p->ntet)) || (rc = dalloc(&p->d_fix, p->P)) ||
        (rc = dalloc(&p->d_restvol, p->ntet)) || (rc = dalloc(&p->d_guide, std::max<size_t>(1, p->guide.size()))) ||
        (rc = dalloc(&p->d_coords, C * 6 * p->P)) || (rc = dalloc(&p->d_ssd, C * p->ntet * 2)) ||
        (rc = dalloc(&p->d_cov, C * p->ntet * 2)) || (rc = dalloc(&p->d_def, C * p->ntet)) ||
        (rc = dalloc(&p->d_fold, C * p->ntet)) || (rc = dalloc(&p->d_loc, C * 2 * std::max(1, p->ng))) ||
        (rc = dalloc(&p->d_gterm, C * 2 * std::max(1, p->ng))) || (rc = dalloc(&p->d_sums, C * 4)) ||
        (rc = dalloc(&p->d_samples, 2)) || (rc = dalloc(&p->d_prob, 1)) || (rc = dalloc(&p->d_obj, C * 4)))
      goto fail_;
    if (!p->gs_id.empty()) {
      if ((rc = dalloc(&p->d_gs_id, p->gs_id.size())) || (rc = dalloc(&p->d_gs_ptr, p->gs_ptr.size())) ||
          (rc = dalloc(&p->d_gs_mem, p->gs_mem.size())))
        goto fail_;
      cudaMemcpyAsync(p->d_gs_id, p->gs_id.data(), sizeof(int) * p->gs_id.size(), cudaMemcpyHostToDevice, p->st);
      cudaMemcpyAsync(p->d_gs_ptr, p->gs_ptr.data(), sizeof(int) * p->gs_ptr.size(), cudaMemcpyHostToDevice, p->st);
      cudaMemcpyAsync(p->d_gs_mem, p->gs_mem.data(), sizeof(int) * p->gs_mem.size(), cudaMemcpyHostToDevice, p->st);
    }
    cudaMemcpyAsync(p->d_tet, t4.data(), sizeof(int4) * p->ntet, cudaMemcpyHostToDevice, p->st);
    cudaMemcpyAsync(p->d_fperm, p->fperm.data(), sizeof(uint32_t) * p->ntet, cudaMemcpyHostToDevice, p->st);
    cudaMemcpyAsync(p->d_fix, p->fixmask.data(), p->P, cudaMemcpyHostToDevice, p->st);
    cudaMemcpyAsync(p->d_restvol, rv.data(), sizeof(float) * p->ntet, cudaMemcpyHostToDevice, p->st);
    if (p->ng)
      cudaMemcpyAsync(p->d_guide, p->guide.data(), sizeof(double) * p->guide.size(), cudaMemcpyHostToDevice, p->st);
    cudaMemsetAsync(p->d_samples, 0, 2 * sizeof(unsigned long long), p->st);
    DevProblem& h = p->hp;
    memset(&h, 0, sizeof(h));
    for (int k = 0; k < 2; ++k) {
      h.plain[k] = p->plain[k];
      h.cells[k] = p->cells[k];
      h.cflag[k] = p->cflag[k];
      h.cmask[k] = p->cmask[k];
      h.nzsat[k] = p->nzsat[k];
      h.occ[k] = p->occ[k];
      h.occd[k] = p->occd[k];
      for (int a = 0; a < 3; ++a) {
        h.n[k][a] = p->n[k][a];
        h.spd[k][a] = p->sp[k][a];
        h.sp[k][a] = (float)p->sp[k][a];
      }
    }
    h.dtype = p->storage;
    h.P = p->P;
    h.ntet = p->ntet;
    for (int a = 0; a < 3; ++a) h.m[a] = p->m[a];
    h.tet = p->d_tet;
    h.fperm = p->d_fperm;
    h.fixmask = p->d_fix;
    h.star_ptr = p->d_star_ptr;
    h.star = p->d_star;
    h.rest_vol = p->d_restvol;
    h.black_rule = p->black_rule;
    h.model = p->model;
    h.lam = (float)p->lam;
    h.mu = (float)p->mu;
    h.sim_norm = (double)p->n[0][0] * p->n[0][1] * p->n[0][2] + (double)p->n[1][0] * p->n[1][1] * p->n[1][2];
    h.def_norm = p->model == DMR_LINEAR ? rvs : 10.0 * p->ntet;
    h.guid_norm = 2.0 * std::max(1, p->ng);
    h.ng = p->ng;
    h.guide = p->d_guide;
    h.gsid = p->d_gs_id;
    h.gptr = p->d_gs_ptr;
    h.gmem = p->d_gs_mem;
    h.C = 0;
    h.coords = p->d_coords;
    h.c_ssd = p->d_ssd;
    h.c_cov = p->d_cov;
    h.c_def = p->d_def;
    h.c_fold = p->d_fold;
    h.c_loc = p->d_loc;
    h.c_gterm = p->d_gterm;
    h.sums = p->d_sums;
    h.samples = p->d_samples;
    h.executed = p->d_samples + 1;
    if ((rc = upload_prob(p))) goto fail_;
    cudaError_t e = cudaStreamSynchronize(p->st);
    if (e != cudaSuccess) {
      rc = fail(DMR_ECUDA, std::string("create: ") + cudaGetErrorString(e));
      goto fail_;
    }
  }
  *out = p;
  return DMR_OK;
fail_:
  release_problem(p);
  delete p;
  return rc;
}

int dmr_problem_destroy(dmr_problem* p) {
  if (!p) return DMR_OK;
  cudaStreamSynchronize(p->st);
  if (p->st2) {
    cudaStreamSynchronize(p->st2);
    cudaStreamDestroy(p->st2);
  }
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  release_problem(p);
  delete p;
  return DMR_OK;
}

int dmr_set_stream(dmr_problem* p, void* stream) {
  if (!p) return fail(DMR_EINVAL, "null problem");
  p->st = (cudaStream_t)stream;
  return DMR_OK;
}

int dmr_problem_info(const dmr_problem* p, int* n_points, int* n_tets) {
  if (!p) return fail(DMR_EINVAL, "null problem");
  if (n_points) *n_points = p->P;
  if (n_tets) *n_tets = p->ntet;
  return DMR_OK;
}

int dmr_tets_out(const dmr_problem* p, int* tets) {
  if (!p || !tets) return fail(DMR_EINVAL, "null argument");
  memcpy(tets, p->tets.data(), sizeof(int) * 4 * (size_t)p->ntet);
  return DMR_OK;
}

int dmr_set_tile(dmr_problem* p, int warps_per_cta, int voxels_per_warp) {
  if (!p) return fail(DMR_EINVAL, "null problem");
  if (warps_per_cta == 0) warps_per_cta = 8;
  if (voxels_per_warp == 0) voxels_per_warp = 32;
  if (warps_per_cta != 4 && warps_per_cta != 8 && warps_per_cta != 16) return fail(DMR_EINVAL, "warps_per_cta");
  if (voxels_per_warp != 32 && voxels_per_warp != 64 && voxels_per_warp != 128) return fail(DMR_EINVAL, "voxels_per_warp");
  p->warps = warps_per_cta;
  p->vpw = voxels_per_warp;
  return DMR_OK;
}

int dmr_get_tile(const dmr_problem* p, int* w, int* v) {
  if (!p) return fail(DMR_EINVAL, "null problem");
  if (w) *w = p->warps;
  if (v) *v = p->vpw;
  return DMR_OK;
}

// ------------------------------------------------------------ FOS
int dmr_set_fos(dmr_problem* p, int n_groups, const int* group_ptr, const int* group_pts) {
  if (!p || n_groups < 1 || !group_ptr || !group_pts) return fail(DMR_EINVAL, "bad FOS arguments");
  if (group_ptr[0] != 0) return fail(DMR_EINVAL, "group_ptr[0] must be 0");
  std::vector<int> gp(group_ptr, group_ptr + n_groups + 1);
  int gmax = 0;
  for (int g = 0; g < n_groups; ++g) {
    int sz = gp[g + 1] - gp[g];
    if (sz < 1 || sz > 254) return fail(DMR_EINVAL, "group sizes must be 1..254");
    gmax = std::max(gmax, sz);
  }
  std::vector<int> pts(group_pts, group_pts + gp[n_groups]);
  for (int v : pts)
    if (v < 0 || v >= p->P) return fail(DMR_EINVAL, "group point id out of range");
  // touched sets and per-vertex slots
  std::vector<int> tptr(n_groups + 1, 0), tl;
  std::vector<uint32_t> slot;
  std::vector<int> mark(p->ntet, -1);
  int maxt = 0;
  for (int g = 0; g < n_groups; ++g) {
    std::vector<int> ts;
    for (int j = gp[g]; j < gp[g + 1]; ++j) {
      int v = pts[j];
      for (int q = gp[g]; q < j; ++q)
        if (pts[q] == v) return fail(DMR_EINVAL, "duplicate point in a group");
      for (int s = p->star_ptr[v]; s < p->star_ptr[v + 1]; ++s)
        if (mark[p->star[s]] != g) {
          mark[p->star[s]] = g;
          ts.push_back(p->star[s]);
        }
    }
    std::sort(ts.begin(), ts.end());
    for (int t : ts) {
      uint32_t sl = 0;
      for (int i = 0; i < 4; ++i) {
        int v = p->tets[4 * (size_t)t + i];
        for (int j = gp[g]; j < gp[g + 1]; ++j)
          if (pts[j] == v) sl |= (uint32_t)(j - gp[g] + 1) << (8 * i);
      }
      tl.push_back(t);
      slot.push_back(sl);
    }
    tptr[g + 1] = (int)tl.size();
    maxt = std::max(maxt, (int)ts.size());
  }
  // greedy colouring: groups in one wave touch disjoint tets
  std::vector<int> color(n_groups, -1), tet_last(p->ntet, -1);
  std::vector<std::vector<int>> waves;
  std::vector<std::vector<char>> used;  // per wave: tets used
  for (int g = 0; g < n_groups; ++g) {
    int w = 0;
    for (;; ++w) {
      if (w == (int)waves.size()) {
        waves.emplace_back();
        used.emplace_back(p->ntet, 0);
      }
      bool ok = true;
      for (int j = tptr[g]; j < tptr[g + 1] && ok; ++j)
        if (used[w][tl[j]]) ok = false;
      if (ok) break;
    }
    for (int j = tptr[g]; j < tptr[g + 1]; ++j) used[w][tl[j]] = 1;
    waves[w].push_back(g);
    color[g] = w;
  }
  p->wave_ptr.assign(1, 0);
  p->wave_groups.clear();
  for (auto& w : waves) {
    p->wave_groups.insert(p->wave_groups.end(), w.begin(), w.end());
    p->wave_ptr.push_back((int)p->wave_groups.size());
  }
  p->n_groups = n_groups;
  p->gmax = gmax;
  p->max_touched = maxt;
  p->g_ptr = gp;
  p->g_pts = pts;
  p->g_tptr = tptr;
  p->g_tets = tl;
  p->g_slot = slot;
  dfree(p->d_gptr);
  dfree(p->d_gpts);
  int rc;
  if ((rc = dalloc(&p->d_gptr, gp.size())) || (rc = dalloc(&p->d_gpts, pts.size()))) return rc;
  CU(cudaMemcpyAsync(p->d_gptr, gp.data(), sizeof(int) * gp.size(), cudaMemcpyHostToDevice, p->st));
  CU(cudaMemcpyAsync(p->d_gpts, pts.data(), sizeof(int) * pts.size(), cudaMemcpyHostToDevice, p->st));
  CU(cudaStreamSynchronize(p->st));
  p->have_partial = false;
  clear_layouts(p);  // group ids now mean other groups
  return DMR_OK;
}

int dmr_fos_info(const dmr_problem* p, int* max_group, int* max_touched, int* n_waves) {
  if (!p) return fail(DMR_EINVAL, "null problem");
  if (p->n_groups == 0) return fail(DMR_ESTATE, "no FOS registered");
  if (max_group) *max_group = p->gmax;
  if (max_touched) *max_touched = p->max_touched;
  if (n_waves) *n_waves = (int)p->wave_ptr.size() - 1;
  return DMR_OK;
}

int dmr_fos_waves(const dmr_problem* p, int* wave_ptr, int* wave_groups) {
  if (!p) return fail(DMR_EINVAL, "null problem");
  if (p->n_groups == 0) return fail(DMR_ESTATE, "no FOS registered");
  if (wave_ptr) memcpy(wave_ptr, p->wave_ptr.data(), sizeof(int) * p->wave_ptr.size());
  if (wave_groups) memcpy(wave_groups, p->wave_groups.data(), sizeof(int) * p->wave_groups.size());
  return DMR_OK;
}

// ------------------------------------------------------------ evaluation
namespace {

Batch make_batch(dmr_problem* p, Scratch& s, int n_tt, int n_tr) {
  Batch b;
  memset(&b, 0, sizeof(b));
  b.n_tt = n_tt;
  b.tt_trial = s.tt_trial;
  b.tt_tet = s.tt_tet;
  b.tt_slot = s.tt_slot;
  b.n_trials = n_tr;
  b.tr_prob = nullptr;
  b.tr_cand = s.tr_cand;
  b.tr_first = s.tr_first;
  b.tr_ntt = s.tr_ntt;
  b.tr_coords = s.tr_coords;
  b.gmax = std::max(1, p->gmax);
  b.rec = s.rec;
  b.o_ssd = s.o_ssd;
  b.o_cov = s.o_cov;
  b.o_def = s.o_def;
  b.o_fold = s.o_fold;
  b.work = s.work;
  b.slow = s.slow;
  b.aff_cap = s.aff_cap;
  b.aff_n = p->ng > 0 ? s.aff_n : nullptr;
  b.aff_idx = s.aff_idx;
  b.aff_loc = s.aff_loc;
  b.aff_term = s.aff_term;
  b.tr_delta = s.tr_delta;
  b.tr_obj = s.tr_obj;
  return b;
}

// The batch of a cached eval_partial layout: lists from the layout, outputs
// and records in the problem's scratch.
Batch layout_batch(dmr_problem* p, Layout* L, int n_tr) {
  Batch b = make_batch(p, p->sc, L->tot, n_tr);
  b.tt_trial = L->tt_trial;
  b.tt_tet = L->tt_tet;
  b.tt_slot = L->tt_slot;
  b.tr_cand = L->tr_cand;
  b.tr_first = L->tr_first;
  b.tr_ntt = L->tr_ntt;
  return b;
}

}  // namespace

int dmr_eval_full(dmr_problem* p, int n_cand, const double* coords, double* obj_out) {
  if (!p || !coords || !obj_out) return fail(DMR_EINVAL, "null argument");
  if (n_cand < 1 || n_cand > p->cap) return fail(DMR_EINVAL, "n_cand out of range");
  p->have_partial = false;
  size_t csz = (size_t)6 * p->P;
  CU(cudaMemcpyAsync(p->d_coords, coords, sizeof(double) * csz * n_cand, cudaMemcpyDefault, p->st));
  p->C = n_cand;
  p->hp.C = n_cand;
  int rc;
  if ((rc = upload_prob(p))) return rc;
  const int chunk_tt_cap = 1 << 20;
  int cpc = std::max(1, std::min(n_cand, chunk_tt_cap / std::max(1, p->ntet)));
  if ((rc = p->sc.ensure(cpc * p->ntet, cpc, std::max(1, p->gmax), 2 * std::max(1, p->ng)))) return rc;
  std::vector<int> tt_trial((size_t)cpc * p->ntet), tt_tet((size_t)cpc * p->ntet), tr_cand(cpc), tr_first(cpc),
      tr_ntt(cpc);
  for (int c0 = 0; c0 < n_cand; c0 += cpc) {
    int nc = std::min(cpc, n_cand - c0);
    for (int ci = 0; ci < nc; ++ci) {
      tr_cand[ci] = c0 + ci;
      tr_first[ci] = ci * p->ntet;
      tr_ntt[ci] = p->ntet;
      for (int t = 0; t < p->ntet; ++t) {
        tt_trial[(size_t)ci * p->ntet + t] = ci;
        tt_tet[(size_t)ci * p->ntet + t] = t;
      }
    }
    int ntt = nc * p->ntet;
    CU(cudaMemcpyAsync(p->sc.tt_trial, tt_trial.data(), sizeof(int) * ntt, cudaMemcpyHostToDevice, p->st));
    CU(cudaMemcpyAsync(p->sc.tt_tet, tt_tet.data(), sizeof(int) * ntt, cudaMemcpyHostToDevice, p->st));
    CU(cudaMemcpyAsync(p->sc.tr_cand, tr_cand.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, p->st));
    CU(cudaMemcpyAsync(p->sc.tr_first, tr_first.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, p->st));
    CU(cudaMemcpyAsync(p->sc.tr_ntt, tr_ntt.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, p->st));
    Batch b = make_batch(p, p->sc, ntt, nc);
    b.tt_slot = nullptr;
    b.tr_coords = nullptr;
    size_t off = (size_t)c0 * p->ntet;
    b.o_ssd = p->d_ssd + 2 * off;
    b.o_cov = p->d_cov + 2 * off;
    b.o_def = p->d_def + off;
    b.o_fold = p->d_fold + off;
    launch_setup(p->d_prob, b, p->st);
    launch_raster(p->d_prob, b, p->storage, p->warps, p->vpw, p->n_sm, p->st);
    if (p->ng > 0) launch_locate_full(p->d_prob, p->hp, b, c0, nc, p->st);
    launch_reduce_full(p->d_prob, c0, nc, b, p->d_obj + 4 * (size_t)c0, p->st);
    CU(cudaGetLastError());
    // host staging arrays are reused by the next chunk
    CU(cudaStreamSynchronize(p->st));
  }
  bool host_dst;
  if ((rc = copy_out(obj_out, p->d_obj, sizeof(double) * 4 * n_cand, p->st, host_dst))) return rc;
  if (host_dst) CU(cudaStreamSynchronize(p->st));
  return DMR_OK;
}

int dmr_eval_partial(dmr_problem* p, int n_trials, const int* group_ids, const int* cand_ids,
                     const double* trial_coords, double* obj_out) {
  if (!p || !group_ids || !cand_ids || !trial_coords || !obj_out) return fail(DMR_EINVAL, "null argument");
  if (p->n_groups == 0) return fail(DMR_ESTATE, "no FOS registered");
  if (p->C == 0) return fail(DMR_ESTATE, "no population (call dmr_eval_full first)");
  if (n_trials < 1) return fail(DMR_EINVAL, "n_trials must be >= 1");
  std::vector<int> gid(n_trials), cid(n_trials);
  if (is_device_ptr(group_ids)) CU(cudaMemcpy(gid.data(), group_ids, sizeof(int) * n_trials, cudaMemcpyDeviceToHost));
  else std::memcpy(gid.data(), group_ids, sizeof(int) * n_trials);
  if (is_device_ptr(cand_ids)) CU(cudaMemcpy(cid.data(), cand_ids, sizeof(int) * n_trials, cudaMemcpyDeviceToHost));
  else std::memcpy(cid.data(), cand_ids, sizeof(int) * n_trials);
  const cudaStream_t st = p->st;
  int rc;
  Layout* L = nullptr;
  for (Layout* c : p->layouts)
    if (c->gid == gid && c->cid == cid) {
      if (c->max_cid >= p->C) return fail(DMR_EINVAL, "candidate id out of range");
      L = c;
      break;
    }
  if (!L) {
    std::vector<int> first(n_trials), ntt(n_trials);
    long tot = 0;
    for (int k = 0; k < n_trials; ++k) {
      if (gid[k] < 0 || gid[k] >= p->n_groups) return fail(DMR_EINVAL, "group id out of range");
      if (cid[k] < 0 || cid[k] >= p->C) return fail(DMR_EINVAL, "candidate id out of range");
      first[k] = (int)tot;
      ntt[k] = p->g_tptr[gid[k] + 1] - p->g_tptr[gid[k]];
      tot += ntt[k];
    }
    if (tot > (1L << 30)) return fail(DMR_EINVAL, "too many trial tets");
    std::vector<int> tt_trial(tot), tt_tet(tot);
    std::vector<uint32_t> tt_slot(tot);
    for (int k = 0; k < n_trials; ++k) {
      int g = gid[k];
      for (int j = 0; j < ntt[k]; ++j) {
        tt_trial[first[k] + j] = k;
        tt_tet[first[k] + j] = p->g_tets[p->g_tptr[g] + j];
        tt_slot[first[k] + j] = p->g_slot[p->g_tptr[g] + j];
      }
    }
    // commit safety: accepted trials of a candidate must touch disjoint tets
    std::vector<int> order(n_trials);
    for (int k = 0; k < n_trials; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cid[a] < cid[b]; });
    std::vector<int> cptr(1, 0), ctr;
    bool safe = true;
    {
      std::vector<int> stamp(p->ntet, -1);
      int prev = -1, ci = -1;
      for (int idx : order) {
        if (cid[idx] != prev) {
          prev = cid[idx];
          ++ci;
          if (ci > 0) cptr.push_back((int)ctr.size());
        }
        ctr.push_back(idx);
        int g = gid[idx];
        for (int j = p->g_tptr[g]; j < p->g_tptr[g + 1]; ++j) {
          int t = p->g_tets[j];
          if (stamp[t] == cid[idx]) safe = false;
          stamp[t] = cid[idx];
        }
      }
      cptr.push_back((int)ctr.size());
    }
    if ((int)p->layouts.size() >= kLayoutCache) {
      // evict the least recently used layout (cudaFree waits for its users)
      auto it = std::min_element(p->layouts.begin(), p->layouts.end(),
                                 [](const Layout* x, const Layout* y) { return x->used < y->used; });
      (*it)->release();
      delete *it;
      p->layouts.erase(it);
    }
    L = new Layout();
    L->gid = gid;
    L->cid = cid;
    L->first = std::move(first);
    L->ntt = std::move(ntt);
    L->cptr = std::move(cptr);
    L->ctr = std::move(ctr);
    L->tot = (int)tot;
    L->safe = safe;
    L->max_cid = *std::max_element(cid.begin(), cid.end());
    if ((rc = dalloc(&L->tt_trial, (size_t)std::max(1L, tot))) || (rc = dalloc(&L->tt_tet, (size_t)std::max(1L, tot))) ||
        (rc = dalloc(&L->tt_slot, (size_t)std::max(1L, tot))) || (rc = dalloc(&L->tr_cand, n_trials)) ||
        (rc = dalloc(&L->tr_group, n_trials)) || (rc = dalloc(&L->tr_first, n_trials)) ||
        (rc = dalloc(&L->tr_ntt, n_trials)) || (rc = dalloc(&L->cand_ptr, L->cptr.size())) ||
        (rc = dalloc(&L->cand_trials, std::max<size_t>(1, L->ctr.size())))) {
      L->release();
      delete L;
      return rc;
    }
    // the host vectors live as long as the layout, so the copies may stay in flight
    CU(cudaMemcpyAsync(L->tt_trial, tt_trial.data(), sizeof(int) * tot, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(L->tt_tet, tt_tet.data(), sizeof(int) * tot, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(L->tt_slot, tt_slot.data(), sizeof(uint32_t) * tot, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(L->tr_cand, L->cid.data(), sizeof(int) * n_trials, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(L->tr_group, L->gid.data(), sizeof(int) * n_trials, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(L->tr_first, L->first.data(), sizeof(int) * n_trials, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(L->tr_ntt, L->ntt.data(), sizeof(int) * n_trials, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(L->cand_ptr, L->cptr.data(), sizeof(int) * L->cptr.size(), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(L->cand_trials, L->ctr.data(), sizeof(int) * L->ctr.size(), cudaMemcpyHostToDevice, st));
    // tt_* are pageable temporaries: their copies are staged before the calls return
    p->layouts.push_back(L);
  }
  L->used = ++p->layout_clock;
  p->cur = L;
  const long tot = L->tot;
  const bool safe = L->safe;
  if ((rc = p->sc.ensure((int)tot, n_trials, p->gmax, 2 * std::max(1, p->ng)))) return rc;
  CU(cudaMemcpyAsync(p->sc.tr_coords, trial_coords, sizeof(double) * 6 * p->gmax * (size_t)n_trials, cudaMemcpyDefault,
                     st));
  Batch b = layout_batch(p, L, n_trials);
  launch_setup(p->d_prob, b, st);
  if (p->ng > 0 && !p->st2) {
    CU(cudaStreamCreateWithFlags(&p->st2, cudaStreamNonBlocking));
    CU(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming));
  }
  // landmark relocation needs only the set-up records: it runs on a side
  // stream beside the raster kernels that complete deferred work
  launch_raster(p->d_prob, b, p->storage, p->warps, p->vpw, p->n_sm, st, p->ng > 0 ? p->st2 : nullptr,
                p->ev_fork);
  if (p->ng > 0) {
    launch_landmarks_partial(p->d_prob, b, p->st2);
    CU(cudaEventRecord(p->ev_join, p->st2));
    CU(cudaStreamWaitEvent(st, p->ev_join, 0));
  }
  launch_reduce_partial(p->d_prob, b, st);
  CU(cudaGetLastError());
  bool host_dst;
  if ((rc = copy_out(obj_out, p->sc.tr_obj, sizeof(double) * 4 * n_trials, st, host_dst))) return rc;
  if (host_dst) CU(cudaStreamSynchronize(st));
  p->have_partial = true;
  p->partial_safe = safe;
  p->last_ntr = n_trials;
  p->last_ntt = (int)tot;
  p->last_cand = L->cid;
  p->last_group = L->gid;
  p->last_first = L->first;
  p->last_ntt_v = L->ntt;
  p->last_nlist = (int)L->cptr.size() - 1;
  return DMR_OK;
}

namespace {

int do_commit(dmr_problem* p, const uint8_t* d_accept) {
  Batch b = layout_batch(p, p->cur, p->last_ntr);
  launch_commit(p->d_prob, b, d_accept, p->cur->tr_group, p->d_gptr, p->d_gpts, p->cur->cand_ptr,
                p->cur->cand_trials, p->last_nlist, p->st);
  CU(cudaGetLastError());
  p->have_partial = false;
  return DMR_OK;
}

}  // namespace

int dmr_commit(dmr_problem* p, const uint8_t* accept) {
  if (!p || !accept) return fail(DMR_EINVAL, "null argument");
  if (!p->have_partial) return fail(DMR_ESTATE, "no partial evaluation to commit");
  if (!is_device_ptr(accept)) {
    // disjointness of accepted trials per candidate
    std::vector<int> stamp(p->ntet, -1);
    std::vector<int> order;
    for (int k = 0; k < p->last_ntr; ++k)
      if (accept[k]) order.push_back(k);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return p->last_cand[a] < p->last_cand[b]; });
    for (int k : order) {
      int g = p->last_group[k];
      for (int j = p->g_tptr[g]; j < p->g_tptr[g + 1]; ++j) {
        int t = p->g_tets[j];
        if (stamp[t] == p->last_cand[k]) return fail(DMR_EINVAL, "accepted trials of one candidate overlap");
        stamp[t] = p->last_cand[k];
      }
    }
  }
  CU(cudaMemcpyAsync(p->sc.accept, accept, p->last_ntr, cudaMemcpyDefault, p->st));
  int rc = do_commit(p, p->sc.accept);
  if (rc) return rc;
  CU(cudaStreamSynchronize(p->st));
  return DMR_OK;
}

int dmr_commit_improving(dmr_problem* p, uint8_t* accept_out) {
  if (!p) return fail(DMR_EINVAL, "null problem");
  if (!p->have_partial) return fail(DMR_ESTATE, "no partial evaluation to commit");
  if (!p->partial_safe) return fail(DMR_EINVAL, "trials of one candidate overlap; commit explicitly");
  Batch b = layout_batch(p, p->cur, p->last_ntr);
  launch_accept(p->d_prob, b, p->sc.accept, p->st);
  int ntr = p->last_ntr;
  int rc = do_commit(p, p->sc.accept);
  if (rc) return rc;
  if (accept_out) {
    bool host_dst;
    if ((rc = copy_out(accept_out, p->sc.accept, ntr, p->st, host_dst))) return rc;
    if (host_dst) CU(cudaStreamSynchronize(p->st));
  }
  return DMR_OK;
}

int dmr_objectives_out(dmr_problem* p, int n, const int* cand_ids, double* out) {
  if (!p || !cand_ids || !out) return fail(DMR_EINVAL, "null argument");
  std::vector<int> cid(std::max(n, 1));
  CU(cudaMemcpy(cid.data(), cand_ids, sizeof(int) * n, cudaMemcpyDefault));
  std::vector<double> raw(4 * (size_t)p->cap), res(4 * (size_t)std::max(n, 1));
  CU(cudaMemcpyAsync(raw.data(), p->d_sums, sizeof(double) * 4 * std::max(p->C, 1), cudaMemcpyDeviceToHost, p->st));
  CU(cudaStreamSynchronize(p->st));
  for (int k = 0; k < n; ++k) {
    if (cid[k] < 0 || cid[k] >= p->C) return fail(DMR_EINVAL, "candidate id out of range");
    const double* s = &raw[4 * (size_t)cid[k]];
    res[4 * k + 0] = s[0] / p->hp.sim_norm;
    res[4 * k + 1] = s[1] / p->hp.def_norm;
    res[4 * k + 2] = p->ng > 0 ? s[2] / p->hp.guid_norm : 0.0;
    res[4 * k + 3] = s[3];
  }
  CU(cudaMemcpy(out, res.data(), sizeof(double) * 4 * n, cudaMemcpyDefault));
  return DMR_OK;
}

int dmr_coords_out(dmr_problem* p, int cand, double* out) {
  if (!p || !out) return fail(DMR_EINVAL, "null argument");
  if (cand < 0 || cand >= p->C) return fail(DMR_EINVAL, "candidate id out of range");
  CU(cudaStreamSynchronize(p->st));
  CU(cudaMemcpy(out, p->d_coords + (size_t)cand * 6 * p->P, sizeof(double) * 6 * p->P, cudaMemcpyDefault));
  return DMR_OK;
}

int dmr_terms_out(dmr_problem* p, int cand, int* cov, double* ssd, double* def, int* fold) {
  if (!p) return fail(DMR_EINVAL, "null problem");
  if (cand < 0 || cand >= p->C) return fail(DMR_EINVAL, "candidate id out of range");
  CU(cudaStreamSynchronize(p->st));
  size_t off = (size_t)cand * p->ntet;
  if (cov) CU(cudaMemcpy(cov, p->d_cov + 2 * off, sizeof(int) * 2 * p->ntet, cudaMemcpyDefault));
  if (ssd) CU(cudaMemcpy(ssd, p->d_ssd + 2 * off, sizeof(double) * 2 * p->ntet, cudaMemcpyDefault));
  if (def) CU(cudaMemcpy(def, p->d_def + off, sizeof(double) * p->ntet, cudaMemcpyDefault));
  if (fold) CU(cudaMemcpy(fold, p->d_fold + off, sizeof(int) * p->ntet, cudaMemcpyDefault));
  return DMR_OK;
}

int dmr_landmarks_out(dmr_problem* p, int cand, int* loc, double* term) {
  if (!p) return fail(DMR_EINVAL, "null problem");
  if (cand < 0 || cand >= p->C) return fail(DMR_EINVAL, "candidate id out of range");
  if (p->ng == 0) return DMR_OK;
  CU(cudaStreamSynchronize(p->st));
  size_t off = (size_t)cand * 2 * p->ng;
  if (loc) CU(cudaMemcpy(loc, p->d_loc + off, sizeof(int) * 2 * p->ng, cudaMemcpyDefault));
  if (term) CU(cudaMemcpy(term, p->d_gterm + off, sizeof(double) * 2 * p->ng, cudaMemcpyDefault));
  return DMR_OK;
}

int dmr_trial_out(dmr_problem* p, int k, int* tets, int* cov, double* ssd, double* def, int* fold) {
  if (!p) return fail(DMR_EINVAL, "null problem");
  if (p->last_group.empty()) return fail(DMR_ESTATE, "no partial evaluation");
  if (k < 0 || k >= p->last_ntr) return fail(DMR_EINVAL, "trial index out of range");
  CU(cudaStreamSynchronize(p->st));
  int f = p->last_first[k], n = p->last_ntt_v[k];
  int g = p->last_group[k];
  if (tets) memcpy(tets, &p->g_tets[p->g_tptr[g]], sizeof(int) * n);
  if (cov) CU(cudaMemcpy(cov, p->sc.o_cov + 2 * (size_t)f, sizeof(int) * 2 * n, cudaMemcpyDefault));
  if (ssd) CU(cudaMemcpy(ssd, p->sc.o_ssd + 2 * (size_t)f, sizeof(double) * 2 * n, cudaMemcpyDefault));
  if (def) CU(cudaMemcpy(def, p->sc.o_def + f, sizeof(double) * n, cudaMemcpyDefault));
  if (fold) CU(cudaMemcpy(fold, p->sc.o_fold + f, sizeof(int) * n, cudaMemcpyDefault));
  return n;
}

int dmr_link_check(dmr_problem* p, int n_cand, const int* cand_ids, int* out) {
  if (!p || !cand_ids || !out) return fail(DMR_EINVAL, "null argument");
  if (n_cand < 1 || n_cand > p->C) return fail(DMR_EINVAL, "n_cand out of range");
  std::vector<int> cid(n_cand);
  if (is_device_ptr(cand_ids)) CU(cudaMemcpy(cid.data(), cand_ids, sizeof(int) * n_cand, cudaMemcpyDeviceToHost));
  else std::memcpy(cid.data(), cand_ids, sizeof(int) * n_cand);
  for (int c : cid)
    if (c < 0 || c >= p->C) return fail(DMR_EINVAL, "candidate id out of range");
  int* d_c = nullptr;
  int* d_out = nullptr;
  int rc;
  if ((rc = dalloc(&d_c, n_cand)) || (rc = dalloc(&d_out, 2 * (size_t)n_cand))) {
    dfree(d_c);
    return rc;
  }
  cudaMemcpyAsync(d_c, cid.data(), sizeof(int) * n_cand, cudaMemcpyHostToDevice, p->st);
  cudaMemsetAsync(d_out, 0, sizeof(int) * 2 * n_cand, p->st);
  launch_link_check(p->d_prob, p->hp, d_c, n_cand, d_out, p->st);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_out, sizeof(int) * 2 * n_cand, cudaMemcpyDefault, p->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
  dfree(d_c);
  dfree(d_out);
  if (e != cudaSuccess) return fail(DMR_ECUDA, std::string("link check: ") + cudaGetErrorString(e));
  return DMR_OK;
}

int dmr_refine(const double* coarse, int n_cand, const int* m, double* fine, void* stream) {
  if (!coarse || !fine || !m || n_cand < 0) return fail(DMR_EINVAL, "refine: null argument");
  for (int a = 0; a < 3; ++a)
    if (m[a] < 2 || m[a] > 1024) return fail(DMR_EINVAL, "refine: points per axis out of range");
  if (n_cand == 0) return DMR_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t P = (size_t)m[0] * m[1] * m[2];
  const size_t PF = (size_t)(2 * m[0] - 1) * (2 * m[1] - 1) * (2 * m[2] - 1);
  const size_t nc = (size_t)n_cand * 6 * P, nf = (size_t)n_cand * 6 * PF;
  const double* dc = coarse;
  double* df = fine;
  double *tc = nullptr, *tf = nullptr;
  int rc = DMR_OK;
  if (!is_device_ptr(coarse)) {
    if ((rc = dalloc(&tc, nc))) return rc;
    cudaMemcpyAsync(tc, coarse, sizeof(double) * nc, cudaMemcpyHostToDevice, st);
    dc = tc;
  }
  const bool host_out = !is_device_ptr(fine);
  if (host_out) {
    if ((rc = dalloc(&tf, nf))) {
      dfree(tc);
      return rc;
    }
    df = tf;
  }
  launch_refine(dc, n_cand, m, df, st);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && host_out) e = cudaMemcpyAsync(fine, tf, sizeof(double) * nf, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  dfree(tc);
  dfree(tf);
  if (e != cudaSuccess) return fail(DMR_ECUDA, std::string("refine: ") + cudaGetErrorString(e));
  return DMR_OK;
}

int dmr_sample_counts(dmr_problem* p, long long* counted, long long* executed, int reset) {
  if (!p || (!counted && !executed)) return fail(DMR_EINVAL, "null argument");
  unsigned long long v[2] = {0, 0};
  CU(cudaMemcpyAsync(v, p->d_samples, sizeof(v), cudaMemcpyDeviceToHost, p->st));
  CU(cudaStreamSynchronize(p->st));
  if (counted) *counted = (long long)v[0];
  if (executed) *executed = (long long)v[1];
  if (reset) CU(cudaMemsetAsync(p->d_samples, 0, sizeof(v), p->st));
  return DMR_OK;
}

int dmr_samples(dmr_problem* p, long long* samples, int reset) { return dmr_sample_counts(p, samples, nullptr, reset); }

// ------------------------------------------------------------ autotuner
int dmr_autotune(dmr_problem* p, int n_cand, int* best_warps, int* best_vpw, float* ms_table) {
  if (!p) return fail(DMR_EINVAL, "null problem");
  if (p->C == 0) return fail(DMR_ESTATE, "no population (call dmr_eval_full first)");
  int nc = n_cand > 0 ? std::min(n_cand, p->C) : std::min(p->C, 16);
  int rc;
  if ((rc = p->sc.ensure(nc * p->ntet, nc, std::max(1, p->gmax), 2 * std::max(1, p->ng)))) return rc;
  std::vector<int> tt_trial((size_t)nc * p->ntet), tt_tet((size_t)nc * p->ntet), tr_cand(nc), tr_first(nc), tr_ntt(nc);
  for (int ci = 0; ci < nc; ++ci) {
    tr_cand[ci] = ci;
    tr_first[ci] = ci * p->ntet;
    tr_ntt[ci] = p->ntet;
    for (int t = 0; t < p->ntet; ++t) {
      tt_trial[(size_t)ci * p->ntet + t] = ci;
      tt_tet[(size_t)ci * p->ntet + t] = t;
    }
  }
  int ntt = nc * p->ntet;
  cudaStream_t st = p->st;
  CU(cudaMemcpyAsync(p->sc.tt_trial, tt_trial.data(), sizeof(int) * ntt, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(p->sc.tt_tet, tt_tet.data(), sizeof(int) * ntt, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(p->sc.tr_cand, tr_cand.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(p->sc.tr_first, tr_first.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(p->sc.tr_ntt, tr_ntt.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, st));
  Batch b = make_batch(p, p->sc, ntt, nc);
  b.tt_slot = nullptr;
  b.tr_coords = nullptr;
  launch_setup(p->d_prob, b, st);
  const int W[3] = {4, 8, 16}, V[3] = {32, 64, 128};
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  float best = 3.0e38f;
  int bw = p->warps, bv = p->vpw;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      float tot = 0.f;
      for (int rep = 0; rep < 4; ++rep) {
        cudaMemsetAsync(b.work, 0, 3 * sizeof(unsigned), st);
        cudaEventRecord(e0, st);
        launch_raster(p->d_prob, b, p->storage, W[i], V[j], p->n_sm, st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) tot += ms;  // first launch warms up
      }
      float ms = tot / 3.f;
      if (ms_table) ms_table[3 * i + j] = ms;
      if (ms < best) {
        best = ms;
        bw = W[i];
        bv = V[j];
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CU(cudaGetLastError());
  p->warps = bw;
  p->vpw = bv;
  if (best_warps) *best_warps = bw;
  if (best_vpw) *best_vpw = bv;
  return DMR_OK;
}

// ------------------------------------------------------------ generation plan
int dmr_plan_destroy(dmr_plan* pl) {
  if (!pl) return DMR_OK;
  if (pl->p) cudaStreamSynchronize(pl->p->st);
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  for (cudaEvent_t e : pl->ev) cudaEventDestroy(e);
  dfree(pl->tt_trial); dfree(pl->tt_tet); dfree(pl->tt_slot); dfree(pl->tr_cand); dfree(pl->tr_first);
  dfree(pl->tr_ntt); dfree(pl->tr_group); dfree(pl->tr_prob); dfree(pl->deltas); dfree(pl->cand_ptr);
  dfree(pl->cand_trials);
  dfree(pl->slot_q); dfree(pl->slot_src);
  for (double*& r : pl->raw) dfree(r);
  if (pl->d_raw) cudaFree((void*)pl->d_raw);
  dfree(pl->d_rawG);
  pl->sc.release();
  delete pl;
  return DMR_OK;
}

namespace {

// One generation of partial evaluations for one or more problems, captured
// into a CUDA graph.  Wave w of the plan holds wave w of every problem that
// has one; trials are ordered (problem, candidate, group).  deltas[q] is the
// host copy [n_groups][n_cand][2][3][G_q] of problem q.
int build_plan(const std::vector<dmr_problem*>& probs, const DevProblem* d_probs, const int* d_gptr,
               const int* d_gpts, const std::vector<int>& goff, const std::vector<std::vector<int>>& cands,
               const std::vector<std::vector<double>>& deltas, dmr_plan** out) {
  dmr_problem* p0 = probs[0];
  const int nq = (int)probs.size();
  int G = 1, nw = 0, acap = 2;
  for (dmr_problem* p : probs) {
    G = std::max(G, p->gmax);
    nw = std::max(nw, (int)p->wave_ptr.size() - 1);
    acap = std::max(acap, 2 * p->ng);
  }
  dmr_plan* pl = new (std::nothrow) dmr_plan();
  if (!pl) return fail(DMR_ENOMEM, "host allocation failed");
  pl->p = p0;
  std::vector<int> tt_trial, tt_tet, tr_cand, tr_first, tr_ntt, tr_group, tr_prob, cptr, ctr;
  std::vector<uint32_t> tt_slot;
  std::vector<double> dl;
  std::vector<int> sl_q;
  std::vector<long long> sl_src;
  std::vector<int> w_tt0, w_ntt, w_tr0, w_ntr, w_c0, w_nlist;
  int max_tt = 0, max_tr = 0;
  const size_t dl_per = (size_t)6 * G;
  for (int w = 0; w < nw; ++w) {
    w_tt0.push_back((int)tt_trial.size());
    w_tr0.push_back((int)tr_cand.size());
    w_c0.push_back((int)cptr.size());
    int k = 0, ttw = 0, nlist = 0;
    for (int q = 0; q < nq; ++q) {
      dmr_problem* p = probs[q];
      if (w >= (int)p->wave_ptr.size() - 1) continue;
      const int Gq = p->gmax;
      const int nc = (int)cands[q].size();
      // trials group-major (every candidate of a group, then the next group):
      // consecutive raster items then sample the same image region, which
      // stays in L2 across the candidates; each candidate's trial list (for
      // the sums) keeps its groups in wave order
      const int ng_w = p->wave_ptr[w + 1] - p->wave_ptr[w];
      for (int ci = 0; ci < nc; ++ci) {
        cptr.push_back((int)ctr.size() - w_tr0.back());  // position in this wave's list
        ++nlist;
        for (int j = 0; j < ng_w; ++j) ctr.push_back(k + j * nc + ci);
      }
      for (int gi = p->wave_ptr[w]; gi < p->wave_ptr[w + 1]; ++gi) {
        for (int ci = 0; ci < nc; ++ci, ++k) {
          const int g = p->wave_groups[gi];
          tr_cand.push_back(cands[q][ci]);
          tr_group.push_back(goff[q] + g);
          tr_prob.push_back(q);
          tr_first.push_back(ttw);
          const int n = p->g_tptr[g + 1] - p->g_tptr[g];
          tr_ntt.push_back(n);
          for (int j = 0; j < n; ++j) {
            tt_trial.push_back(k);
            tt_tet.push_back(p->g_tets[p->g_tptr[g] + j]);
            tt_slot.push_back(p->g_slot[p->g_tptr[g] + j]);
          }
          ttw += n;
          // [2][3][Gq] of the problem -> [2][3][G] of the plan
          const double* src = &deltas[q][((size_t)g * nc + ci) * 6 * Gq];
          sl_q.push_back(q);
          sl_src.push_back((long long)(((size_t)g * nc + ci) * 6 * Gq));
          size_t base = dl.size();
          dl.resize(base + dl_per, 0.0);
          for (int ma = 0; ma < 6; ++ma)
            for (int j = 0; j < Gq; ++j) dl[base + (size_t)ma * G + j] = src[(size_t)ma * Gq + j];
        }
      }
    }
    cptr.push_back(k);
    w_ntt.push_back(ttw);
    w_ntr.push_back(k);
    w_nlist.push_back(nlist);
    max_tt = std::max(max_tt, ttw);
    max_tr = std::max(max_tr, k);
  }
  int rc;
  if ((rc = dalloc(&pl->tt_trial, tt_trial.size())) || (rc = dalloc(&pl->tt_tet, tt_tet.size())) ||
      (rc = dalloc(&pl->tt_slot, tt_slot.size())) || (rc = dalloc(&pl->tr_cand, tr_cand.size())) ||
      (rc = dalloc(&pl->tr_first, tr_first.size())) || (rc = dalloc(&pl->tr_ntt, tr_ntt.size())) ||
      (rc = dalloc(&pl->tr_group, tr_group.size())) || (rc = dalloc(&pl->tr_prob, tr_prob.size())) ||
      (rc = dalloc(&pl->deltas, dl.size())) || (rc = dalloc(&pl->cand_ptr, cptr.size())) ||
      (rc = dalloc(&pl->cand_trials, ctr.size())) || (rc = pl->sc.ensure(max_tt, max_tr, G, acap)) ||
      (rc = dalloc(&pl->slot_q, std::max<size_t>(1, sl_q.size()))) ||
      (rc = dalloc(&pl->slot_src, std::max<size_t>(1, sl_src.size())))) {
    dmr_plan_destroy(pl);
    return rc;
  }
  pl->G = G;
  pl->n_slots = (int)sl_q.size();
  for (int q = 0; q < nq; ++q) {
    pl->raw_count.push_back(deltas[q].size());
    pl->raw_G.push_back(probs[q]->gmax);
  }
  auto up = [&](void* d, const void* h, size_t bytes) { return cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice); };
  if (up(pl->tt_trial, tt_trial.data(), 4 * tt_trial.size()) || up(pl->tt_tet, tt_tet.data(), 4 * tt_tet.size()) ||
      up(pl->tt_slot, tt_slot.data(), 4 * tt_slot.size()) || up(pl->tr_cand, tr_cand.data(), 4 * tr_cand.size()) ||
      up(pl->tr_first, tr_first.data(), 4 * tr_first.size()) || up(pl->tr_ntt, tr_ntt.data(), 4 * tr_ntt.size()) ||
      up(pl->tr_group, tr_group.data(), 4 * tr_group.size()) || up(pl->tr_prob, tr_prob.data(), 4 * tr_prob.size()) ||
      up(pl->deltas, dl.data(), 8 * dl.size()) || up(pl->cand_ptr, cptr.data(), 4 * cptr.size()) ||
      up(pl->cand_trials, ctr.data(), 4 * ctr.size()) || up(pl->slot_q, sl_q.data(), 4 * sl_q.size()) ||
      up(pl->slot_src, sl_src.data(), 8 * sl_src.size())) {
    dmr_plan_destroy(pl);
    return fail(DMR_ECUDA, "plan upload failed");
  }
  pl->ev.assign(2 * (size_t)nw, nullptr);
  for (auto& e : pl->ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      dmr_plan_destroy(pl);
      return fail(DMR_ECUDA, "event create failed");
    }
  bool any_ng = false;
  for (dmr_problem* p : probs) any_ng = any_ng || p->ng > 0;
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    dmr_plan_destroy(pl);
    return fail(DMR_ECUDA, "stream create failed");
  }
  // side branch of the graph: landmark relocation needs only the set-up
  // records, so it runs beside the raster kernels
  cudaStream_t cs2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_sums = nullptr;
  if (cudaStreamCreateWithFlags(&cs2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ev_sums, cudaEventDisableTiming) != cudaSuccess) {
    if (cs2) cudaStreamDestroy(cs2);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (ev_sums) cudaEventDestroy(ev_sums);
    cudaStreamDestroy(cs);
    dmr_plan_destroy(pl);
    return fail(DMR_ECUDA, "stream create failed");
  }
  for (dmr_problem* p : probs) cudaStreamSynchronize(p->st);
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  int launches = 0;
  for (int w = 0; w < nw && e == cudaSuccess; ++w) {
    Batch b = make_batch(p0, pl->sc, w_ntt[w], w_ntr[w]);
    b.tt_trial = pl->tt_trial + w_tt0[w];
    b.tt_tet = pl->tt_tet + w_tt0[w];
    b.tt_slot = pl->tt_slot + w_tt0[w];
    b.tr_cand = pl->tr_cand + w_tr0[w];
    b.tr_first = pl->tr_first + w_tr0[w];
    b.tr_ntt = pl->tr_ntt + w_tr0[w];
    b.tr_prob = pl->tr_prob + w_tr0[w];
    b.gmax = G;
    b.aff_cap = pl->sc.aff_cap;
    b.aff_n = any_ng ? pl->sc.aff_n : nullptr;
    const int* trg = pl->tr_group + w_tr0[w];
    launch_propose(d_probs, b, trg, d_gptr, d_gpts, pl->deltas + (size_t)w_tr0[w] * dl_per, cs);
    launch_setup(d_probs, b, cs);
    cudaEventRecordWithFlags(pl->ev[2 * w], cs, cudaEventRecordExternal);
    launch_raster(d_probs, b, p0->storage, p0->warps, p0->vpw, p0->n_sm, cs, any_ng ? cs2 : nullptr,
                  any_ng ? ev_fork : nullptr);
    cudaEventRecordWithFlags(pl->ev[2 * w + 1], cs, cudaEventRecordExternal);
    launches += 2 + kRasterLaunches;
    if (any_ng) {
      // the fork is recorded inside launch_raster before the fast kernel
      launch_landmarks_partial(d_probs, b, cs2);
      cudaEventRecord(ev_join, cs2);
      cudaStreamWaitEvent(cs, ev_join, 0);
      ++launches;
    }
    // with guidance points the side stream orders the sums of wave w before
    // the next wave's landmark kernel (which rewrites the delta buffer), and
    // the next wave's reduce waits for that landmark kernel
    launch_reduce_commit(d_probs, b, pl->sc.accept, trg, d_gptr, d_gpts, pl->cand_ptr + w_c0[w],
                         pl->cand_trials + w_tr0[w], w_nlist[w], cs, any_ng ? cs2 : nullptr,
                         any_ng ? ev_sums : nullptr);
    launches += 2;
    e = cudaGetLastError();
  }
  if (any_ng) {
    cudaEventRecord(ev_join, cs2);
    cudaStreamWaitEvent(cs, ev_join, 0);
  }
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(cs);
  cudaStreamDestroy(cs2);
  cudaEventDestroy(ev_fork);
  cudaEventDestroy(ev_join);
  cudaEventDestroy(ev_sums);
  if (e != cudaSuccess || e2 != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    dmr_plan_destroy(pl);
    return fail(DMR_ECUDA, std::string("graph capture failed: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  pl->graph = g;
  e = cudaGraphInstantiate(&pl->exec, g, 0);
  if (e != cudaSuccess) {
    dmr_plan_destroy(pl);
    return fail(DMR_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  pl->launches = launches;
  for (dmr_problem* p : probs) p->have_partial = false;
  *out = pl;
  return DMR_OK;
}

int check_cands(dmr_problem* p, int n_cand, const int* cand_ids, std::vector<int>& cid) {
  if (p->n_groups == 0) return fail(DMR_ESTATE, "no FOS registered");
  if (p->C == 0) return fail(DMR_ESTATE, "no population (call dmr_eval_full first)");
  if (n_cand < 1 || n_cand > p->C) return fail(DMR_EINVAL, "n_cand out of range");
  cid.resize(n_cand);
  CU(cudaMemcpy(cid.data(), cand_ids, sizeof(int) * n_cand, cudaMemcpyDefault));
  std::vector<int> s(cid);
  std::sort(s.begin(), s.end());
  for (int k = 0; k < n_cand; ++k) {
    if (s[k] < 0 || s[k] >= p->C) return fail(DMR_EINVAL, "candidate id out of range");
    if (k && s[k] == s[k - 1]) return fail(DMR_EINVAL, "duplicate candidate id");
  }
  return DMR_OK;
}

}  // namespace

int dmr_plan_generation(dmr_problem* p, int n_cand, const int* cand_ids, const double* deltas, dmr_plan** out) {
  if (!p || !cand_ids || !deltas || !out) return fail(DMR_EINVAL, "null argument");
  *out = nullptr;
  std::vector<int> cid;
  int rc = check_cands(p, n_cand, cand_ids, cid);
  if (rc) return rc;
  std::vector<std::vector<double>> hd(1, std::vector<double>((size_t)p->n_groups * n_cand * 6 * p->gmax));
  CU(cudaMemcpy(hd[0].data(), deltas, sizeof(double) * hd[0].size(), cudaMemcpyDefault));
  return build_plan({p}, p->d_prob, p->d_gptr, p->d_gpts, {0}, {cid}, hd, out);
}

struct dmr_batch {
  std::vector<dmr_problem*> probs;
  DevProblem* d_probs = nullptr;
  int* d_gptr = nullptr;
  int* d_gpts = nullptr;
  std::vector<int> goff;
};

int dmr_batch_create(int n, dmr_problem* const* probs, dmr_batch** out) {
  if (!probs || !out || n < 1) return fail(DMR_EINVAL, "bad batch arguments");
  *out = nullptr;
  for (int q = 0; q < n; ++q) {
    if (!probs[q]) return fail(DMR_EINVAL, "null problem in batch");
    if (probs[q]->storage != probs[0]->storage) return fail(DMR_EINVAL, "problems of a batch share one storage dtype");
    if (probs[q]->dev != probs[0]->dev) return fail(DMR_EINVAL, "problems of a batch share one device");
    if (probs[q]->n_groups == 0) return fail(DMR_ESTATE, "every problem of a batch needs a FOS");
  }
  dmr_batch* bt = new (std::nothrow) dmr_batch();
  if (!bt) return fail(DMR_ENOMEM, "host allocation failed");
  bt->probs.assign(probs, probs + n);
  std::vector<DevProblem> hp(n);
  std::vector<int> gptr(1, 0), gpts;
  for (int q = 0; q < n; ++q) {
    dmr_problem* p = probs[q];
    hp[q] = p->hp;
    bt->goff.push_back((int)gptr.size() - 1);
    for (int g = 0; g < p->n_groups; ++g) {
      for (int j = p->g_ptr[g]; j < p->g_ptr[g + 1]; ++j) gpts.push_back(p->g_pts[j]);
      gptr.push_back((int)gpts.size());
    }
  }
  int rc;
  if ((rc = dalloc(&bt->d_probs, n)) || (rc = dalloc(&bt->d_gptr, gptr.size())) || (rc = dalloc(&bt->d_gpts, gpts.size()))) {
    dfree(bt->d_probs);
    dfree(bt->d_gptr);
    dfree(bt->d_gpts);
    delete bt;
    return rc;
  }
  cudaMemcpy(bt->d_probs, hp.data(), sizeof(DevProblem) * n, cudaMemcpyHostToDevice);
  cudaMemcpy(bt->d_gptr, gptr.data(), sizeof(int) * gptr.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(bt->d_gpts, gpts.data(), sizeof(int) * gpts.size(), cudaMemcpyHostToDevice);
  *out = bt;
  return DMR_OK;
}

int dmr_batch_destroy(dmr_batch* bt) {
  if (!bt) return DMR_OK;
  for (dmr_problem* p : bt->probs) cudaStreamSynchronize(p->st);
  dfree(bt->d_probs);
  dfree(bt->d_gptr);
  dfree(bt->d_gpts);
  delete bt;
  return DMR_OK;
}

int dmr_batch_plan_generation(dmr_batch* bt, const int* n_cand, const int* const* cand_ids,
                              const double* const* deltas, dmr_plan** out) {
  if (!bt || !n_cand || !cand_ids || !deltas || !out) return fail(DMR_EINVAL, "null argument");
  *out = nullptr;
  const int nq = (int)bt->probs.size();
  std::vector<std::vector<int>> cands(nq);
  std::vector<std::vector<double>> hd(nq);
  for (int q = 0; q < nq; ++q) {
    dmr_problem* p = bt->probs[q];
    if (!cand_ids[q] || !deltas[q]) return fail(DMR_EINVAL, "null per-problem argument");
    int rc = check_cands(p, n_cand[q], cand_ids[q], cands[q]);
    if (rc) return rc;
    hd[q].resize((size_t)p->n_groups * n_cand[q] * 6 * p->gmax);
    CU(cudaMemcpy(hd[q].data(), deltas[q], sizeof(double) * hd[q].size(), cudaMemcpyDefault));
  }
  return build_plan(bt->probs, bt->d_probs, bt->d_gptr, bt->d_gpts, bt->goff, cands, hd, out);
}

int dmr_plan_update(dmr_plan* pl, const double* const* deltas) {
  if (!pl || !pl->exec || !deltas) return fail(DMR_EINVAL, "null argument");
  const int nq = (int)pl->raw_count.size();
  cudaStream_t st = pl->p->st;
  if (pl->raw.empty()) {
    pl->raw.assign(nq, nullptr);
    for (int q = 0; q < nq; ++q) {
      int rc = dalloc(&pl->raw[q], std::max<size_t>(1, pl->raw_count[q]));
      if (rc) return rc;
    }
    CU(cudaMalloc((void**)&pl->d_raw, sizeof(double*) * nq));
    int rc = dalloc(&pl->d_rawG, nq);
    if (rc) return rc;
    CU(cudaMemcpy(pl->d_rawG, pl->raw_G.data(), sizeof(int) * nq, cudaMemcpyHostToDevice));
  }
  std::vector<const double*> src(nq);
  for (int q = 0; q < nq; ++q) {
    if (!deltas[q]) return fail(DMR_EINVAL, "null deltas");
    if (is_device_ptr(deltas[q])) {
      src[q] = deltas[q];
    } else {
      CU(cudaMemcpyAsync(pl->raw[q], deltas[q], sizeof(double) * pl->raw_count[q], cudaMemcpyHostToDevice, st));
      src[q] = pl->raw[q];
    }
  }
  // pageable host memory: both copies are staged before the calls return
  CU(cudaMemcpyAsync((void*)pl->d_raw, src.data(), sizeof(double*) * nq, cudaMemcpyHostToDevice, st));
  launch_gather_deltas(pl->d_raw, pl->slot_q, pl->slot_src, pl->d_rawG, pl->n_slots, pl->G, pl->deltas, st);
  CU(cudaGetLastError());
  return DMR_OK;
}

int dmr_plan_run(dmr_plan* pl) {
  if (!pl || !pl->exec) return fail(DMR_EINVAL, "null plan");
  CU(cudaGraphLaunch(pl->exec, pl->p->st));
  return DMR_OK;
}

int dmr_plan_kernel_ms(const dmr_plan* pl, float* setup_ms, float* raster_ms) {
  if (!pl) return fail(DMR_EINVAL, "null plan");
  float ra = 0.f;
  for (size_t w = 0; w + 1 < pl->ev.size(); w += 2) {
    float b = 0.f;
    CU(cudaEventElapsedTime(&b, pl->ev[w], pl->ev[w + 1]));
    ra += b;
  }
  if (setup_ms) *setup_ms = -1.f;
  if (raster_ms) *raster_ms = ra;
  return DMR_OK;
}

int dmr_plan_launches(const dmr_plan* pl, int* launches) {
  if (!pl || !launches) return fail(DMR_EINVAL, "null argument");
  *launches = pl->launches;
  return DMR_OK;
}

}  // extern "C"
