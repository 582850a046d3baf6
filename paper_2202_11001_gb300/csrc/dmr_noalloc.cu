// dmr_eval_one_noalloc: full evaluation of one candidate that allocates no
// memory.  Its scratch (geometry records, per-tet terms, landmark terms and
// the sums) lives in one file-scope device array of fixed size that the
// library holds on every device that loads it, until the process exits.
//
// Who needs it: callers that must not call cudaMalloc/cudaFree at the point
// of evaluation -- latency-critical optimiser loops (cudaMalloc/cudaFree
// synchronise the device and can stall for milliseconds), and hosts whose
// device memory is fully reserved by another allocator (a framework's caching
// allocator that owns the whole budget, or a memory pool sized up front), so
// that a library-side cudaMalloc would fail or evict the caller's data.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <string>

#include "../../include/dmr.h"
#include "dmr_internal.cuh"

using namespace dmr;

namespace {

constexpr int kMaxTets = 4608;   // meshes up to 10 x 10 x 10 points (4374 tets)
constexpr int kMaxGuide = 512;   // guidance pairs

constexpr size_t al(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffProb = 0;
constexpr size_t kOffRec = al(kOffProb + sizeof(DevProblem));
constexpr size_t kOffSsd = al(kOffRec + 2 * (size_t)kMaxTets * sizeof(ItemRec));
constexpr size_t kOffCov = al(kOffSsd + 2 * (size_t)kMaxTets * sizeof(double));
constexpr size_t kOffDef = al(kOffCov + 2 * (size_t)kMaxTets * sizeof(int));
constexpr size_t kOffFold = al(kOffDef + (size_t)kMaxTets * sizeof(double));
constexpr size_t kOffTtTrial = al(kOffFold + (size_t)kMaxTets * sizeof(int));
constexpr size_t kOffTtTet = al(kOffTtTrial + (size_t)kMaxTets * sizeof(int));
constexpr size_t kOffTrial = al(kOffTtTet + (size_t)kMaxTets * sizeof(int));   // cand, first, ntt
constexpr size_t kOffLoc = al(kOffTrial + 3 * sizeof(int));
constexpr size_t kOffGterm = al(kOffLoc + 2 * (size_t)kMaxGuide * sizeof(int));
constexpr size_t kOffSums = al(kOffGterm + 2 * (size_t)kMaxGuide * sizeof(double));
constexpr size_t kOffSlow = al(kOffSums + 4 * sizeof(double));
constexpr size_t kOffCount = al(kOffSlow + 2 * (size_t)kMaxTets * sizeof(int));  // samples, executed (u64), work (3 x u32)
constexpr size_t kScratchBytes = al(kOffCount + 32);

// The scratch.  Host code must not pass this name to a kernel: on the host it
// is only a stand-in; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
unsigned char* g_addr[kMaxDevices] = {nullptr};

int err(int code, const std::string& m) { return set_error(code, m); }

// Fill what the shared kernels read and zero what they accumulate into.
__global__ void k_noalloc_init(DevProblem hp, unsigned char* base, int ntet) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    *(DevProblem*)(base + kOffProb) = hp;
    int* tr = (int*)(base + kOffTrial);
    tr[0] = 0;     // candidate 0 of the scratch problem
    tr[1] = 0;     // first (trial, tet) pair
    tr[2] = ntet;  // all tets
    ((unsigned long long*)(base + kOffCount))[0] = 0ull;
    ((unsigned long long*)(base + kOffCount))[1] = 0ull;
    for (int k = 0; k < 3; ++k) ((unsigned*)(base + kOffCount + 16))[k] = 0u;
  }
  if (i < ntet) {
    ((int*)(base + kOffTtTrial))[i] = 0;
    ((int*)(base + kOffTtTet))[i] = i;
  }
}

}  // namespace

// Declared in include/dmr.h.
extern "C" int dmr_eval_one_noalloc(dmr_problem* p, const double* coords, double* obj_out) {
  if (!p || !coords || !obj_out) return err(DMR_EINVAL, "dmr_eval_one_noalloc: null argument");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return err(DMR_ECUDA, "dmr_eval_one_noalloc: no current device");
  // the scratch address is per device: the problem's kernels run on the
  // problem's device, so that device must be the current one
  if (problem_device_id(p) != dev)
    return err(DMR_EINVAL, "dmr_eval_one_noalloc: the problem was created on device " +
                               std::to_string(problem_device_id(p)) + ", the current device is " + std::to_string(dev));
  cudaPointerAttributes a1, a2;
  if (cudaPointerGetAttributes(&a1, coords) != cudaSuccess || cudaPointerGetAttributes(&a2, obj_out) != cudaSuccess ||
      (a1.type != cudaMemoryTypeDevice && a1.type != cudaMemoryTypeManaged) ||
      (a2.type != cudaMemoryTypeDevice && a2.type != cudaMemoryTypeManaged)) {
    cudaGetLastError();
    return err(DMR_EINVAL, "dmr_eval_one_noalloc: coords and obj_out must be device pointers");
  }
  DevProblem hp;
  int storage = 0, warps = 8, n_sm = 1;
  cudaStream_t st = nullptr;
  if (problem_view(p, &hp, &storage, &warps, &n_sm, &st) != DMR_OK)
    return err(DMR_EINVAL, "dmr_eval_one_noalloc: bad problem");
  if (hp.ntet > kMaxTets)
    return err(DMR_EINVAL, "dmr_eval_one_noalloc: mesh has " + std::to_string(hp.ntet) + " tets; the limit is " +
                               std::to_string(kMaxTets));
  if (hp.ng > kMaxGuide)
    return err(DMR_EINVAL, "dmr_eval_one_noalloc: " + std::to_string(hp.ng) + " guidance pairs; the limit is " +
                               std::to_string(kMaxGuide));
  // set-up, once per device, with that device current
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) {
        cudaGetLastError();
        return err(DMR_ECUDA, std::string("dmr_eval_one_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
      g_addr[dev] = (unsigned char*)ptr;
    }
    base = g_addr[dev];
  }
  // the scratch problem: shared images and topology, candidate 0 = coords,
  // caches and sums in the scratch array
  hp.C = 1;
  hp.coords = const_cast<double*>(coords);
  hp.c_ssd = (double*)(base + kOffSsd);
  hp.c_cov = (int*)(base + kOffCov);
  hp.c_def = (double*)(base + kOffDef);
  hp.c_fold = (int*)(base + kOffFold);
  hp.c_loc = (int*)(base + kOffLoc);
  hp.c_gterm = (double*)(base + kOffGterm);
  hp.sums = (double*)(base + kOffSums);
  hp.samples = (unsigned long long*)(base + kOffCount);
  hp.executed = (unsigned long long*)(base + kOffCount) + 1;
  const DevProblem* d_prob = (const DevProblem*)(base + kOffProb);
  Batch b;
  memset(&b, 0, sizeof(b));
  b.n_tt = hp.ntet;
  b.tt_trial = (const int*)(base + kOffTtTrial);
  b.tt_tet = (const int*)(base + kOffTtTet);
  b.tt_slot = nullptr;
  b.n_trials = 1;
  b.tr_prob = nullptr;
  b.tr_cand = (const int*)(base + kOffTrial);
  b.tr_first = (const int*)(base + kOffTrial) + 1;
  b.tr_ntt = (const int*)(base + kOffTrial) + 2;
  b.tr_coords = nullptr;
  b.gmax = 1;
  b.rec = (ItemRec*)(base + kOffRec);
  b.o_ssd = hp.c_ssd;
  b.o_cov = hp.c_cov;
  b.o_def = hp.c_def;
  b.o_fold = hp.c_fold;
  b.work = (unsigned*)(base + kOffCount + 16);
  b.slow = (int*)(base + kOffSlow);
  k_noalloc_init<<<(hp.ntet + 255) / 256, 256, 0, st>>>(hp, base, hp.ntet);
  launch_setup(d_prob, b, st);
  launch_raster(d_prob, b, storage, warps, 32, n_sm, st);
  if (hp.ng > 0) launch_locate_full(d_prob, hp, b, 0, 1, st);
  launch_reduce_full(d_prob, 0, 1, b, obj_out, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return err(DMR_ECUDA, std::string("dmr_eval_one_noalloc: launch: ") + cudaGetErrorString(e));
  return DMR_OK;
}
