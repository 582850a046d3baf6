// Kernels of the GB300 (sm_103a) evaluator for multi-objective dual
// simplex-mesh deformable registration (arXiv 2202.11001).
//
// Precision plan (GB300 runs FP64 at a small fraction of its FP32 rate):
//  * Decisions that must agree exactly with the FP64 definition -- the
//    inside test of a voxel (Sec. 2.3.1 rasterisation with the 3-D top-left
//    tie rule), the fold test (Sec. 2.3.4) and the black-vs-grey test on the
//    mapped coordinate (Sec. 2.3.1) -- are taken in FP32 with a certified
//    error margin; only the rare voxels inside the margin are decided by
//    the FP64 expression itself (explicit _rn intrinsics, no contraction).
//  * Sampling and squared differences run in FP32 with per-lane Kahan sums
//    and an error-free warp reduction; per-tet and per-candidate sums are
//    FP64.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "dmr_internal.cuh"
#include "dmr_device.cuh"

namespace dmr {

// ------------------------------------------------------------ image prep
__global__ void k_convert(const void* src, int sdt, void* dst, int ddt, long n) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float v;
  if (sdt == ST_F32) v = ((const float*)src)[i];
  else if (sdt == ST_BF16) v = __uint_as_float((uint32_t)((const unsigned short*)src)[i] << 16);
  else v = __half2float(((const __half*)src)[i]);
  if (ddt == ST_F32) ((float*)dst)[i] = v;
  else if (ddt == ST_BF16) ((__nv_bfloat16*)dst)[i] = __float2bfloat16_rn(v);
  else ((__half*)dst)[i] = __float2half_rn(v);
}

void launch_convert_image(const void* src, int sdt, void* dst, int ddt, long n, cudaStream_t st) {
  if (n <= 0) return;
  k_convert<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, sdt, dst, ddt, n);
}

__global__ void k_build_cells(const void* plain, int st, int nx, int ny, int nz, void* cells, uint8_t* cflag,
                              unsigned long long* cmask) {
  long Nx = nx + 2, Ny = ny + 2, Nz = nz + 2;
  long id = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (id >= Nx * Ny * Nz) return;
  int i = (int)(id % Nx) - 1, j = (int)((id / Nx) % Ny) - 1, k = (int)(id / (Nx * Ny)) - 1;
  int any0 = 0, all0 = 1;
  uint32_t raw[8];
  float fv[8];
  for (int c = 0; c < 8; ++c) {
    int x = min(max(i + (c & 1), 0), nx - 1);
    int y = min(max(j + ((c >> 1) & 1), 0), ny - 1);
    int z = min(max(k + ((c >> 2) & 1), 0), nz - 1);
    long li = ((long)z * ny + y) * nx + x;
    if (st == ST_F32) {
      fv[c] = ((const float*)plain)[li];
      raw[c] = __float_as_uint(fv[c]);
    } else {
      unsigned short u = ((const unsigned short*)plain)[li];
      raw[c] = u;
      fv[c] = st == ST_BF16 ? __uint_as_float((uint32_t)u << 16) : __half2float(__ushort_as_half(u));
    }
    if (fv[c] == 0.0f) any0 = 1;
    else all0 = 0;
  }
  // 4x4x4 voxel block (i-1 .. i+2 per axis, clamped): every support of a
  // sample whose FP32 cell is this one lies inside it
  int nb_all0 = 1, nb_none0 = 1;
  unsigned long long zm = 0ull;
  for (int dz = -1; dz <= 2; ++dz)
    for (int dy = -1; dy <= 2; ++dy)
      for (int dx = -1; dx <= 2; ++dx) {
        int x = min(max(i + dx, 0), nx - 1), y = min(max(j + dy, 0), ny - 1), z = min(max(k + dz, 0), nz - 1);
        float v = load_plain_dyn(plain, st, ((long)z * ny + y) * nx + x);
        if (v == 0.0f) {
          nb_none0 = 0;
          zm |= 1ull << ((dz + 1) * 16 + (dy + 1) * 4 + (dx + 1));
        } else {
          nb_all0 = 0;
        }
      }
  cmask[id] = zm;
  if (st == ST_F32) {
    // corner pairs along x as (value, difference): the interpolation's first
    // level then needs one FMA per pair (the same FP32 difference)
    float4* p = (float4*)cells + 2 * id;
    p[0] = make_float4(fv[0], fv[1] - fv[0], fv[2], fv[3] - fv[2]);
    p[1] = make_float4(fv[4], fv[5] - fv[4], fv[6], fv[7] - fv[6]);
  } else {
    uint4 w;
    w.x = raw[0] | (raw[1] << 16);
    w.y = raw[2] | (raw[3] << 16);
    w.z = raw[4] | (raw[5] << 16);
    w.w = raw[6] | (raw[7] << 16);
    ((uint4*)cells)[id] = w;
  }
  // bit 4: the cell holds a 0 corner but its block is neither all 0 nor free
  // of 0s, so a sample near a cell face may need more than the corner flags
  const int near = any0 && !nb_all0 && !nb_none0;
  cflag[id] = (uint8_t)(any0 | (all0 << 1) | (nb_all0 << 2) | (nb_none0 << 3) | (near << 4));
}

// Summed-volume table of nonzero voxels: S[z][y][x] = number of nonzero
// voxels with coordinates below (x, y, z) on every axis.  Initialised with the
// indicator shifted by one, then prefix-summed along x, y and z (one thread
// per line).
__global__ void k_nzsat_init(const void* plain, int st, int nx, int ny, int nz, int* S) {
  const long X = nx + 1, Y = ny + 1, Z = nz + 1;
  const long id = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (id >= X * Y * Z) return;
  const int x = (int)(id % X), y = (int)((id / X) % Y), z = (int)(id / (X * Y));
  int v = 0;
  if (x > 0 && y > 0 && z > 0) v = load_plain_dyn(plain, st, ((long)(z - 1) * ny + (y - 1)) * nx + (x - 1)) != 0.0f;
  S[id] = v;
}

__global__ void k_nzsat_scan(int* S, int X, int Y, int Z, int axis) {
  const long id = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long base, stride;
  int len;
  if (axis == 0) {
    if (id >= (long)Y * Z) return;
    base = id * X;
    stride = 1;
    len = X;
  } else if (axis == 1) {
    if (id >= (long)X * Z) return;
    base = (id / X) * X * Y + id % X;
    stride = X;
    len = Y;
  } else {
    if (id >= (long)X * Y) return;
    base = id;
    stride = (long)X * Y;
    len = Z;
  }
  int acc = 0;
  for (int i = 0; i < len; ++i) {
    acc += S[base + i * stride];
    S[base + i * stride] = acc;
  }
}

void launch_build_nzsat(const void* plain, int dtype, const int n[3], int* sat, cudaStream_t st) {
  const int X = n[0] + 1, Y = n[1] + 1, Z = n[2] + 1;
  const long N = (long)X * Y * Z;
  k_nzsat_init<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(plain, dtype, n[0], n[1], n[2], sat);
  const long lines[3] = {(long)Y * Z, (long)X * Z, (long)X * Y};
  for (int a = 0; a < 3; ++a)
    k_nzsat_scan<<<(unsigned)((lines[a] + 127) / 128), 128, 0, st>>>(sat, X, Y, Z, a);
}

// Block occupancy: one thread per 4x4x4 block sets its bit when the block
// holds a nonzero voxel.
__global__ void k_occ(const void* plain, int st, int nx, int ny, int nz, unsigned long long* occ) {
  const int BX = (nx + 3) >> 2, BY = (ny + 3) >> 2, BZ = (nz + 3) >> 2, W = (BX + 63) >> 6;
  const long id = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (id >= (long)BX * BY * BZ) return;
  const int bx = (int)(id % BX), by = (int)((id / BX) % BY), bz = (int)(id / ((long)BX * BY));
  bool any = false;
  for (int z = 4 * bz; z < min(4 * bz + 4, nz) && !any; ++z)
    for (int y = 4 * by; y < min(4 * by + 4, ny) && !any; ++y)
      for (int x = 4 * bx; x < min(4 * bx + 4, nx) && !any; ++x)
        any = load_plain_dyn(plain, st, ((long)z * ny + y) * nx + x) != 0.0f;
  if (any) atomicOr(occ + ((long)bz * BY + by) * W + (bx >> 6), 1ull << (bx & 63));
}

// Dilation by one block: one thread per block ORs the 27 blocks around it.
__global__ void k_occ_dilate(const unsigned long long* occ, int nx, int ny, int nz, unsigned long long* occd) {
  const int BX = (nx + 3) >> 2, BY = (ny + 3) >> 2, BZ = (nz + 3) >> 2, W = (BX + 63) >> 6;
  const long id = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (id >= (long)BX * BY * BZ) return;
  const int bx = (int)(id % BX), by = (int)((id / BX) % BY), bz = (int)(id / ((long)BX * BY));
  bool any = false;
  for (int z = max(bz - 1, 0); z <= min(bz + 1, BZ - 1) && !any; ++z)
    for (int y = max(by - 1, 0); y <= min(by + 1, BY - 1) && !any; ++y)
      for (int x = max(bx - 1, 0); x <= min(bx + 1, BX - 1) && !any; ++x)
        any = (occ[((long)z * BY + y) * W + (x >> 6)] >> (x & 63)) & 1ull;
  if (any) atomicOr(occd + ((long)bz * BY + by) * W + (bx >> 6), 1ull << (bx & 63));
}

void launch_dilate_occ(const unsigned long long* occ, const int n[3], unsigned long long* occd, cudaStream_t st) {
  const long blocks = (long)((n[0] + 3) >> 2) * ((n[1] + 3) >> 2) * ((n[2] + 3) >> 2);
  cudaMemsetAsync(occd, 0, sizeof(unsigned long long) * occ_words(n), st);
  k_occ_dilate<<<(unsigned)((blocks + 127) / 128), 128, 0, st>>>(occ, n[0], n[1], n[2], occd);
}

long occ_words(const int n[3]) {
  const long BX = (n[0] + 3) >> 2, BY = (n[1] + 3) >> 2, BZ = (n[2] + 3) >> 2;
  return BY * BZ * ((BX + 63) >> 6);
}

void launch_build_occ(const void* plain, int dtype, const int n[3], unsigned long long* occ, cudaStream_t st) {
  const long blocks = (long)((n[0] + 3) >> 2) * ((n[1] + 3) >> 2) * ((n[2] + 3) >> 2);
  cudaMemsetAsync(occ, 0, sizeof(unsigned long long) * occ_words(n), st);
  k_occ<<<(unsigned)((blocks + 127) / 128), 128, 0, st>>>(plain, dtype, n[0], n[1], n[2], occ);
}

// Nonzero voxels in the box [q0, q1] (inclusive, inside the image).
static __device__ __forceinline__ long nz_in_box(const int* S, const int* n, const int q0[3], const int q1[3]) {
  const long X = n[0] + 1, XY = X * (n[1] + 1);
  auto at = [&](int x, int y, int z) { return (long)__ldg(S + z * XY + y * X + x); };
  const int x0 = q0[0], y0 = q0[1], z0 = q0[2], x1 = q1[0] + 1, y1 = q1[1] + 1, z1 = q1[2] + 1;
  return at(x1, y1, z1) - at(x0, y1, z1) - at(x1, y0, z1) - at(x1, y1, z0) + at(x0, y0, z1) + at(x0, y1, z0) +
         at(x1, y0, z0) - at(x0, y0, z0);
}

void launch_build_cells(const void* plain, int dtype, const int n[3], void* cells, uint8_t* cflag,
                        unsigned long long* cmask, cudaStream_t st) {
  long N = (long)(n[0] + 2) * (n[1] + 2) * (n[2] + 2);
  k_build_cells<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(plain, dtype, n[0], n[1], n[2], cells, cflag, cmask);
}

// ------------------------------------------------------------ geometry set-up
__device__ __forceinline__ double vcoord(const DevProblem& pr, const Batch& b, int k, int cand, uint32_t slots,
                                         int i, int vid, int mesh, int axis) {
  int sl = (int)((slots >> (8 * i)) & 0xff) - 1;
  if (sl >= 0) return b.tr_coords[(size_t)k * 6 * b.gmax + (size_t)(mesh * 3 + axis) * b.gmax + sl];
  return pr.coords[((size_t)cand * 6 + mesh * 3 + axis) * pr.P + vid];
}

__device__ __forceinline__ float fabs3max(float a, float b, float c) { return fmaxf(fabsf(a), fmaxf(fabsf(b), fabsf(c))); }

// v[i][a] for a runtime vertex index i without indexing local memory
__device__ __forceinline__ double pick4d(const double (&v)[4][3], int i, int a) {
  return i == 0 ? v[0][a] : i == 1 ? v[1][a] : i == 2 ? v[2][a] : v[3][a];
}



// Two threads per (trial, tet), adjacent lanes, thread d for mesh d and
// direction d (Sec. 2.3.1-2.3.4): each loads its mesh's vertices, forms its
// edge vectors, volume and FP32 box, takes the pair's edges, first vertex
// and box by shuffles, and writes its direction's record (its vertices also
// go to the pair's record as the partner's); thread 0 adds the fold counts
// and computes the deformation.  Its roundings of FP64 values to FP32 use
// d2f (integer arithmetic), which leaves the FP64 pipe to the FP64
// arithmetic.
// k_setup writes records as 16-byte words; the layout it relies on
static_assert(offsetof(ItemRec, b0) == 16 && offsetof(ItemRec, b1) == 32 && offsetof(ItemRec, O) == 48 &&
                  offsetof(ItemRec, Op) == 64 && offsetof(ItemRec, cbase) == 80 && offsetof(ItemRec, vr) % 16 == 0 &&
                  offsetof(ItemRec, X) % 16 == 0 && offsetof(ItemRec, XP) % 16 == 0 && sizeof(ItemRec) % 16 == 0,
              "ItemRec layout");

__global__ void __launch_bounds__(128, 4) k_setup(const DevProblem* __restrict__ probs, Batch b) {
  const long gi = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gi == 0 && b.work) b.work[0] = b.work[1] = b.work[2] = 0u;
  const int tt = (int)(gi >> 1), d = (int)(gi & 1);
  if (tt >= b.n_tt) return;  // both lanes of a pair (blocks hold whole pairs)
  const unsigned pair = 3u << (threadIdx.x & 30);
  int k = b.tt_trial[tt];
  int t = b.tt_tet[tt];
  const int pi = b.tr_prob ? b.tr_prob[k] : 0;
  const DevProblem& pr = probs[pi];
  int cand = b.tr_cand[k];
  int4 tv = pr.tet[t];
  int vid[4] = {tv.x, tv.y, tv.z, tv.w};
  uint32_t slots = b.tt_slot ? b.tt_slot[tt] : 0u;
  double own[4][3];
  for (int i = 0; i < 4; ++i)
    for (int a = 0; a < 3; ++a) own[i][a] = vcoord(pr, b, k, cand, slots, i, vid[i], d, a);

  // edge vectors and this mesh's fold (FP64, oracle expression order: the
  // volume sign decides an integer)
  double eo[3][3];
  for (int i = 0; i < 3; ++i)
    for (int a = 0; a < 3; ++a) eo[i][a] = dsub(own[i + 1][a], own[0][a]);
  double r0[3];
  cross3d(eo[1], eo[2], r0);
  const double vol6 = dot3d(eo[0], r0);
  int fold = (vol6 > 0 && isfinite(vol6)) ? 0 : 1;
  // fixed axes: the coordinate must equal its border value exactly; both
  // sides are never 0, so equality is equality of the bit patterns (a NaN
  // differs from every border value either way)
  for (int i = 0; i < 4; ++i) {
    uint8_t fm = pr.fixmask[vid[i]];
    if (!fm) continue;
    int bad = 0;
    for (int a = 0; a < 3; ++a)
      if ((fm >> a) & 1) {
        double rv = ((fm >> (3 + a)) & 1) ? (double)pr.n[d][a] - 0.5 : -0.5;
        if (__double_as_longlong(own[i][a]) != __double_as_longlong(rv)) bad = 1;
      }
    fold += bad;
  }
  fold += __shfl_xor_sync(pair, fold, 1);
  if (d == 0) b.o_fold[tt] = fold;

  // edge differences target - source (direction 0's D; direction 1 uses -D,
  // exactly, since a - b = -(b - a) in round-to-nearest), from the pair's
  // edges
  float Dmf[3][3];
  for (int i = 0; i < 3; ++i)
    for (int a = 0; a < 3; ++a) {
      const double ep = __shfl_xor_sync(pair, eo[i][a], 1);
      Dmf[i][a] = d2f(d == 0 ? dsub(ep, eo[i][a]) : dsub(eo[i][a], ep));
    }
  double par0[3];
  for (int a = 0; a < 3; ++a) par0[a] = __shfl_xor_sync(pair, own[0][a], 1);

  // deformation (FP32 from FP64 edge vectors and their differences)
  double def = 0.0;
  if (d == 0 && pr.model == 0) {
    float es[3][3], dd[3][3];
    for (int i = 0; i < 3; ++i)
      for (int a = 0; a < 3; ++a) {
        es[i][a] = d2f(eo[i][a]);
        dd[i][a] = Dmf[i][a];
      }
    // 6 edges + 4 spokes as combinations of the 3 base edges (v0 at 0):
    // positions 0, e1, e2, e3.  Length change via (lt^2 - ls^2)/(lt + ls).
    const float third = 1.0f / 3.0f;
    float E[10][3], D[10][3];
    for (int a = 0; a < 3; ++a) {
      E[0][a] = es[0][a]; D[0][a] = dd[0][a];
      E[1][a] = es[1][a]; D[1][a] = dd[1][a];
      E[2][a] = es[2][a]; D[2][a] = dd[2][a];
      E[3][a] = es[1][a] - es[0][a]; D[3][a] = dd[1][a] - dd[0][a];
      E[4][a] = es[2][a] - es[0][a]; D[4][a] = dd[2][a] - dd[0][a];
      E[5][a] = es[2][a] - es[1][a]; D[5][a] = dd[2][a] - dd[1][a];
      // spokes: centroid of the opposite face minus the vertex
      E[6][a] = (es[0][a] + es[1][a] + es[2][a]) * third;
      D[6][a] = (dd[0][a] + dd[1][a] + dd[2][a]) * third;
      E[7][a] = (es[1][a] + es[2][a]) * third - es[0][a];
      D[7][a] = (dd[1][a] + dd[2][a]) * third - dd[0][a];
      E[8][a] = (es[0][a] + es[2][a]) * third - es[1][a];
      D[8][a] = (dd[0][a] + dd[2][a]) * third - dd[1][a];
      E[9][a] = (es[0][a] + es[1][a]) * third - es[2][a];
      D[9][a] = (dd[0][a] + dd[1][a]) * third - dd[2][a];
    }
    float acc = 0.0f;
    for (int q = 0; q < 10; ++q) {
      float ls2 = 0.f, lt2 = 0.f, diff2 = 0.f;
      for (int a = 0; a < 3; ++a) {
        float s = E[q][a] * pr.sp[0][a];
        float tt_ = (E[q][a] + D[q][a]) * pr.sp[1][a];
        float dl = fmaf(D[q][a], pr.sp[1][a], E[q][a] * (pr.sp[1][a] - pr.sp[0][a]));  // tt_ - s
        ls2 = fmaf(s, s, ls2);
        lt2 = fmaf(tt_, tt_, lt2);
        diff2 = fmaf(dl, tt_ + s, diff2);
      }
      float den = sqrtf(lt2) + sqrtf(ls2);
      // zero-length edge pairs give 0; non-finite lengths propagate
      float dlen = den > 0.f ? diff2 / den : (den == 0.f ? 0.f : den);
      acc = fmaf(dlen, dlen, acc);
    }
    def = (double)acc;
  }

  // FP32 bounding boxes of the own vertices and, from the pair, of the
  // partner vertices (rounding is monotone, so ceil/floor of the rounded
  // extremes give a superset of the voxels a tet can hold); finiteness of
  // every rounded coordinate
  float olo[3], ohi[3], plo_[3], phi_[3];
  bool ofin = true;
  for (int a = 0; a < 3; ++a) {
    olo[a] = ohi[a] = d2f(own[0][a]);
    ofin = ofin && isfinite(olo[a]);
    for (int i = 1; i < 4; ++i) {
      const float v = d2f(own[i][a]);
      olo[a] = fminf(olo[a], v);
      ohi[a] = fmaxf(ohi[a], v);
      ofin = ofin && isfinite(v);
    }
  }
  for (int a = 0; a < 3; ++a) {
    plo_[a] = __shfl_xor_sync(pair, olo[a], 1);
    phi_[a] = __shfl_xor_sync(pair, ohi[a], 1);
  }
  const bool pfin = __shfl_xor_sync(pair, (int)ofin, 1) != 0;

  // Zero-region bits of the direction (ItemRec::flags bit2 / bit3, kept
  // below only where the map is finite and small): no nonzero / no zero
  // partner voxel within 2 voxels of the partner tet's box (clamped to the
  // image).  A voxel inside the own tet maps into the partner tet (the FP32
  // map within a small fraction of a voxel of it, as for bit1), so its FP32
  // cell and its exact support, clamped, lie in that region: with no nonzero
  // voxel there the sample is 0 and black, with no 0 it is not black.
  int zbits = 0;
  {
    const int* np = pr.n[1 - d];
    if (pfin && pr.nzsat[1 - d]) {
      int q0[3], q1[3];
      for (int a = 0; a < 3; ++a) {
        const float hiv = (float)(np[a] - 1);
        q0[a] = (int)fminf(fmaxf(floorf(plo_[a]) - 2.0f, 0.0f), hiv);
        q1[a] = (int)fminf(fmaxf(ceilf(phi_[a]) + 2.0f, 0.0f), hiv);
      }
      const long nzc = nz_in_box(pr.nzsat[1 - d], np, q0, q1);
      const long vol = (long)(q1[0] - q0[0] + 1) * (q1[1] - q0[1] + 1) * (q1[2] - q0[2] + 1);
      zbits = (nzc == 0 ? 4 : 0) | (nzc == vol ? 8 : 0);
      // bit4 (with bit2): the own image is 0 over the own tet's box too, so
      // every sample is 0 against 0 (d^2 = 0, black or not): only the
      // coverage is counted
      const int* no = pr.n[d];
      if ((zbits & 4) && ofin && pr.nzsat[d]) {
        int o0[3], o1[3];
        bool empty = false;
        for (int a = 0; a < 3; ++a) {
          o0[a] = (int)fminf(fmaxf(ceilf(olo[a]), 0.0f), (float)(no[a] - 1));
          o1[a] = (int)fminf(fmaxf(floorf(ohi[a]), 0.0f), (float)(no[a] - 1));
          empty = empty || o0[a] > o1[a];
        }
        if (!empty && nz_in_box(pr.nzsat[d], no, o0, o1) == 0) zbits |= 16;
      }
    }
  }

  // the direction's record, assembled in registers and written with 16-byte
  // stores
  do {
    ItemRec& R = b.rec[2 * (size_t)tt + d];
    const int* n = pr.n[d];
    const int* np = pr.n[1 - d];
    int flags = (vol6 > 0 && isfinite(vol6)) ? 1 : 0;
    {
      // this thread's mesh is the own mesh of its record and the partner
      // mesh of the pair's record
      double2* xs = reinterpret_cast<double2*>(&R.X[0][0]);
      double2* xp = reinterpret_cast<double2*>(&b.rec[2 * (size_t)tt + (1 - d)].XP[0][0]);
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const int i0 = (2 * q) / 3, a0 = (2 * q) % 3, i1 = (2 * q + 1) / 3, a1 = (2 * q + 1) % 3;
        const double2 v = make_double2(own[i0][a0], own[i1][a1]);
        xs[q] = v;
        xp[q] = v;
      }
    }
    // adjugate rows of the own edge matrix (FP64, fused; they give the face
    // normals below and, rounded, the FP32 map; the decisions that need the
    // exact-order map rebuild it from X and XP); det = 6V_own
    double rr[3][3];
    for (int j = 0; j < 3; ++j) rr[0][j] = r0[j];
    rr[1][0] = fma(eo[2][1], eo[0][2], -eo[2][2] * eo[0][1]);
    rr[1][1] = fma(eo[2][2], eo[0][0], -eo[2][0] * eo[0][2]);
    rr[1][2] = fma(eo[2][0], eo[0][1], -eo[2][1] * eo[0][0]);
    rr[2][0] = fma(eo[0][1], eo[1][2], -eo[0][2] * eo[1][1]);
    rr[2][1] = fma(eo[0][2], eo[1][0], -eo[0][0] * eo[1][2]);
    rr[2][2] = fma(eo[0][0], eo[1][1], -eo[0][1] * eo[1][0]);
    // FP32 map G = [D1 D2 D3][r1; r2; r3] / det from the FP64 edge
    // differences and adjugate rows rounded once: an entry differs from the
    // exact map by at most 8 eps gabs, gabs = max over (c, j) of
    // sum_i |D_ic r_ij| / |det| (>= |G|), which M below takes in place of max |G|
    float G[3][4];
    float gabs = 0.f;
    {
      const float invf = (d == 0 ? 1.0f : -1.0f) / d2f(vol6);
      const float ainv = fabsf(invf);
      float rf[3][3];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) rf[i][j] = d2f(rr[i][j]);
      for (int c = 0; c < 3; ++c)
        for (int j = 0; j < 3; ++j) {
          G[c][j] = fmaf(Dmf[0][c], rf[0][j], fmaf(Dmf[1][c], rf[1][j], Dmf[2][c] * rf[2][j])) * invf;
          const float ga = (fabsf(Dmf[0][c] * rf[0][j]) + fabsf(Dmf[1][c] * rf[1][j]) + fabsf(Dmf[2][c] * rf[2][j])) * ainv;
          gabs = fmaxf(gabs, ga);
        }
    }
    // linear-elastic energy from the source->target map (direction 0)
    if (d == 0 && pr.model == 1 && vol6 != 0.0 && isfinite(vol6)) {
      float H[3][3];
      for (int c = 0; c < 3; ++c)
        for (int j = 0; j < 3; ++j) {
          float g = G[c][j] * pr.sp[1][c] / pr.sp[0][j];
          if (c == j) g += pr.sp[1][c] / pr.sp[0][c] - 1.0f;
          H[c][j] = g;
        }
      float tr = H[0][0] + H[1][1] + H[2][2];
      float ee = 0.f;
      for (int c = 0; c < 3; ++c)
        for (int j = 0; j < 3; ++j) {
          float s = 0.5f * (H[c][j] + H[j][c]);
          ee = fmaf(s, s, ee);
        }
      def = (double)(pr.rest_vol[t] * (pr.mu * ee + 0.5f * pr.lam * tr * tr));
    }
    int4* R4 = reinterpret_cast<int4*>(&R);  // header, b0, b1, O, Op, cbase
    if (!flags) {
      R4[0] = make_int4(0, pi, t, d);
      R4[1] = make_int4(1, 1, 1, 1);
      R4[2] = make_int4(0, 0, 0, 0);
      break;
    }
    // bbox and origins
    const float* lo = olo;
    const float* hi = ohi;
    const float* plo = plo_;
    const float* phi = phi_;
    int O[3], Op[3], B0[3], B1[3];
    int L = 1;
    float La[3];  // per-axis extent: 0 <= q_a <= La - 1 for the box's voxels
    for (int a = 0; a < 3; ++a) {
      float cl = ceilf(lo[a]), fh = floorf(hi[a]);
      B0[a] = cl < 0.f ? 0 : (int)fminf(cl, (float)n[a]);
      B1[a] = fh > (float)(n[a] - 1) ? n[a] - 1 : (int)fmaxf(fh, -1.0f);
      O[a] = (int)fmaxf(fminf(floorf(lo[a]), (float)n[a]), -2.0f);
      Op[a] = (int)fmaxf(fminf(floorf(plo[a]), (float)np[a]), -2.0f);
      L = max(L, B1[a] - O[a] + 1);
      La[a] = (float)max(1, B1[a] - O[a] + 1);
    }
    R4[1] = make_int4(B0[0], B0[1], B0[2], 0);
    R4[2] = make_int4(B1[0], B1[1], B1[2], 0);
    R4[3] = make_int4(O[0], O[1], O[2], 0);
    R4[4] = make_int4(Op[0], Op[1], Op[2], 0);
    if (B0[0] > B1[0] || B0[1] > B1[1] || B0[2] > B1[2]) flags = 0;
    // own vertices relative to O (FP64 difference; FP32 copy for the slices)
    double vd[4][3];
    float V = 0.f;
    for (int i = 0; i < 4; ++i) {
      float vr[3];
      for (int a = 0; a < 3; ++a) {
        vd[i][a] = dsub(own[i][a], i2d(O[a]));
        vr[a] = d2f(vd[i][a]);
        V = fmaxf(V, fabsf(vr[a]));
      }
      *reinterpret_cast<float4*>(&R.vr[i][0]) = make_float4(vr[0], vr[1], vr[2], 0.f);
    }
    // faces: inward FP64 normals from the adjugate rows of the map (for a
    // tet of positive volume, rr[m-1] is the inward normal, with the length
    // of a face cross product, of the face opposite vertex m = 1, 2, 3, and
    // -(rr[0] + rr[1] + rr[2]) that of the face opposite vertex 0; within a
    // few 2^-53 U W of the oracle's normals) and FP64 offsets B = -n.(a - O),
    // each rounded once to FP32.  At a point q = p - O with |q_a| <= La_a
    // on every axis (the box's voxels and the one just outside each row end,
    // the only points the spans evaluate), |A.q| <= aL = sum_a |A_a| La_a,
    // and h(q) = fl(A.q + B) differs from the FP64 predicate by at most
    // eps (aL + |B|) from rounding A and B, plus 3 eps (1 + eps)^3 (aL + |B|)
    // from the three roundings of the evaluation (each partial sum is at most
    // (1 + eps)(aL + |B|); eps = 2^-24), plus 1.5e-14 (U W + an)(L + V) for
    // the FP64 predicate's own rounding (an = sum_a |A_a|, L = max_a La_a).
    // The margin takes 5 eps (aL + |B|) for the FP32 part: a quarter above
    // its bound, which covers the rounding of aL, |B| and of the margin
    // itself.  (The landmark test adds terms in |q| of its own.)
    const double N0[3] = {-((rr[0][0] + rr[1][0]) + rr[2][0]), -((rr[0][1] + rr[1][1]) + rr[2][1]),
                          -((rr[0][2] + rr[1][2]) + rr[2][2])};
    const uint32_t fp = pr.fperm[t];
    const float Lf = (float)L;
    float axf[4];
    // edge magnitudes are bounded by the box extent: |u|, |w| <= ext
    const float ext = 1.001f * fmaxf(hi[0] - lo[0], fmaxf(hi[1] - lo[1], hi[2] - lo[2]));
    const float UW = ext * ext;
    for (int f = 0; f < 4; ++f) {
      const int ia = face_local(fp, f, 0), ib = face_local(fp, f, 1), ic = face_local(fp, f, 2);
      const int opp = 6 - ia - ib - ic;  // the vertex not on face f
      const double nx = opp == 0 ? N0[0] : opp == 1 ? rr[0][0] : opp == 2 ? rr[1][0] : rr[2][0];
      const double ny = opp == 0 ? N0[1] : opp == 1 ? rr[0][1] : opp == 2 ? rr[1][1] : rr[2][1];
      const double nz = opp == 0 ? N0[2] : opp == 1 ? rr[0][2] : opp == 2 ? rr[1][2] : rr[2][2];
      const double Bd = -fma(nx, pick4d(vd, ia, 0), fma(ny, pick4d(vd, ia, 1), nz * pick4d(vd, ia, 2)));
      const float Ax = d2f(nx), Ay = d2f(ny), Az = d2f(nz), Bp = d2f(Bd);
      axf[f] = Ax;
      const float an = fabsf(Ax) + fabsf(Ay) + fabsf(Az);
      const float aL = fabsf(Ax) * La[0] + fabsf(Ay) * La[1] + fabsf(Az) * La[2];
      const float mu = (5.0f / 16777216.0f) * (aL + fabsf(Bp)) + 1.5e-14f * (UW + an) * (Lf + V) + 1e-30f;
      *reinterpret_cast<float4*>(&R.fa[f][0]) = make_float4(Ax, Ay, Az, Bp);
      // fm: margin, 1/A.x, margin growth per voxel of |p - O| (landmarks),
      // and the bound on |A.x - s n_x| beyond FP32 rounding (the fused and
      // the oracle-order FP64 normals differ by a few 2^-53 U W)
      *reinterpret_cast<float4*>(&R.fm[f][0]) = make_float4(
          mu, 1.0f / Ax, (1.0f / 2097152.0f) * an + 1.5e-14f * (UW + an), 3.0e-14f * UW + 1e-30f);
    }
    // FP32 map relative to the origins: p'_rel = vr + G vr + k with
    // k = (O - Op) + d0 + G (O - own_0) in FP32 from the FP64 differences
    // rounded once.  Errors against the exact map at a box voxel v: G's, at
    // most 8 eps gabs per entry (rounding D, r and det, the products and
    // sums, the scaling), enter through G (v - own_0) with |v - own_0| <= L
    // per axis, so at most 8 eps M (M >= 3 gabs L); k's own roundings a few
    // eps M; the evaluation's ~7 eps M: inside the black-decision margin
    // 2^-19 M = 32 eps M
    float gmax = 0.f, kmax = 0.f;
    const float oo0 = d2f(dsub(i2d(O[0]), own[0][0])), oo1 = d2f(dsub(i2d(O[1]), own[0][1])),
                oo2 = d2f(dsub(i2d(O[2]), own[0][2]));
    for (int c = 0; c < 3; ++c) {
      for (int j = 0; j < 3; ++j) gmax = fmaxf(gmax, fabsf(G[c][j]));
      const float d0 = d2f(dsub(par0[c], own[0][c]));
      G[c][3] = ((float)(O[c] - Op[c]) + d0) + fmaf(G[c][0], oo0, fmaf(G[c][1], oo1, G[c][2] * oo2));
      kmax = fmaxf(kmax, fabsf(G[c][3]));
      *reinterpret_cast<float4*>(&R.G[c][0]) = make_float4(G[c][0], G[c][1], G[c][2], G[c][3]);
    }
    float M = (float)L * (1.0f + 3.0f * fmaxf(gmax, gabs)) + kmax + 2.0f;
    // bit1: the partner tet lies within [-0.75, n - 0.25] on every axis and
    // the FP32 map error bound is far below 0.25 voxel, so no mapped voxel
    // coordinate of this tet can leave [-1, n].  fminf/fmaxf skip NaN, so
    // finiteness is checked explicitly: a NaN partner vertex or map entry
    // takes the clamped path.
    bool mapok = M < 4096.0f && pfin;
    for (int c = 0; c < 3; ++c)
      for (int j = 0; j < 4; ++j) mapok = mapok && isfinite(G[c][j]);
    {
      bool in = mapok;
      for (int a = 0; a < 3; ++a) in = in && plo[a] >= -0.75f && phi[a] <= (float)np[a] - 0.25f;
      if (flags && in) flags |= 2;
    }
    if (flags && mapok) flags |= zbits | 32;
    R4[0] = make_int4(flags, pi, t, d);
    // gx: (1 + G00, G10, G20, black-decision margin delta = 2^-19 M)
    *reinterpret_cast<float4*>(&R.gx[0]) = make_float4(1.0f + G[0][0], G[1][0], G[2][0], M * (1.0f / 524288.0f));
    *reinterpret_cast<float4*>(&R.clo[0]) =
        make_float4((float)(-1 - Op[0]), (float)(-1 - Op[1]), (float)(-1 - Op[2]), 0.f);
    *reinterpret_cast<float4*>(&R.chi[0]) =
        make_float4((float)(np[0] - Op[0]), (float)(np[1] - Op[1]), (float)(np[2] - Op[2]), 0.f);
    // corner-cell index: cell (i,j,k) with i = Op.x + floor(p'_rel.x) etc.
    unsigned Sy = (unsigned)(np[0] + 2), Sz = (unsigned)((np[1] + 2) * (np[0] + 2));
    unsigned base = ((unsigned)(Op[2] + 1) * (unsigned)(np[1] + 2) + (unsigned)(Op[1] + 1)) * Sy + (unsigned)(Op[0] + 1);
    base -= (unsigned)MAGIC_BITS * (Sz + Sy + 1u);
    int forder, fshape;
    face_order(axf, forder, fshape);
    R4[5] = make_int4((int)base, forder, fshape, 0);
  } while (false);
  if (d == 0) b.o_def[tt] = def;
}

// ------------------------------------------------------------ refinement
// Grid multi-resolution (Sec. 2.4): one thread per (candidate, mesh, axis,
// fine point).  The corners of the fine point's edge / face / cube are summed
// in halves along its odd axes in z, y, x order, then scaled exactly.
struct RefineDims {
  int m[3], M[3];
  long P, PF;
};

__device__ double refine_corner_sum(const double* v, const RefineDims& d, int A, int B, int C) {
  // up to 8 corners; iterate the odd axes z, y, x as the binary digits of j
  const int oz = C & 1, oy = B & 1, ox = A & 1;
  double s[8];
  int n = 0;
  for (int jz = 0; jz <= oz; ++jz)
    for (int jy = 0; jy <= oy; ++jy)
      for (int jx = 0; jx <= ox; ++jx) {
        const int a = (A - ox) / 2 + jx, b = (B - oy) / 2 + jy, c = (C - oz) / 2 + jz;
        s[n++] = v[a + (long)d.m[0] * (b + (long)d.m[1] * c)];
      }
  // pairwise halves: the last odd axis (x) pairs neighbours first
  for (int w = 1; w < n; w <<= 1)
    for (int i = 0; i + w < n; i += 2 * w) s[i] = dadd(s[i], s[i + w]);
  return s[0];
}

__global__ void k_refine(const double* __restrict__ coarse, int n_cand, RefineDims d, double* __restrict__ fine) {
  const long id = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (id >= (long)n_cand * 6 * d.PF) return;
  const long cma = id / d.PF, q = id % d.PF;
  const int A = (int)(q % d.M[0]), B = (int)((q / d.M[0]) % d.M[1]), C = (int)(q / ((long)d.M[0] * d.M[1]));
  const int k = (A & 1) + (B & 1) + (C & 1);
  const double s = refine_corner_sum(coarse + cma * d.P, d, A, B, C);
  fine[id] = dmul(s, k == 0 ? 1.0 : k == 1 ? 0.5 : k == 2 ? 0.25 : 0.125);
}

void launch_refine(const double* coarse, int n_cand, const int m[3], double* fine, cudaStream_t st) {
  RefineDims d;
  for (int a = 0; a < 3; ++a) {
    d.m[a] = m[a];
    d.M[a] = 2 * m[a] - 1;
  }
  d.P = (long)m[0] * m[1] * m[2];
  d.PF = (long)d.M[0] * d.M[1] * d.M[2];
  const long n = (long)n_cand * 6 * d.PF;
  if (n <= 0) return;
  k_refine<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(coarse, n_cand, d, fine);
}

// ------------------------------------------------------------ link test
// The paper's folding check (Sec. 2.3.4): a point is outside its link (the
// faces of its star's tets that do not contain it) when a ray from it
// crosses the link an even number of times; border points in their plane
// against the star triangles' edges there (2-D), border-edge points between
// their two neighbours along the free axis, corners never.  Ray directions
// (1, kRayY, kRayZ) and (1, kRayY) over the two free axes; triangle crossing
// after Moeller & Trumbore (1997), closed triangle, strictly ahead; segment
// parameter in [0, 1).  FP64 with one rounding per operation, in the
// oracle's order, so the counts equal the oracle's.
constexpr double kRayY = 0.7548776662466927, kRayZ = 0.5698402909980532;

__device__ int ray_hits_triangle(const double* o, const double* a, const double* b, const double* c) {
  const double R[3] = {1.0, kRayY, kRayZ};
  double e1[3], e2[3], tv[3], pv[3], qv[3];
  for (int k = 0; k < 3; ++k) {
    e1[k] = dsub(b[k], a[k]);
    e2[k] = dsub(c[k], a[k]);
    tv[k] = dsub(o[k], a[k]);
  }
  pv[0] = dsub(dmul(R[1], e2[2]), dmul(R[2], e2[1]));
  pv[1] = dsub(dmul(R[2], e2[0]), dmul(R[0], e2[2]));
  pv[2] = dsub(dmul(R[0], e2[1]), dmul(R[1], e2[0]));
  const double det = dadd(dadd(dmul(e1[0], pv[0]), dmul(e1[1], pv[1])), dmul(e1[2], pv[2]));
  if (det == 0.0) return 0;
  const double inv = __ddiv_rn(1.0, det);
  const double u = dmul(dadd(dadd(dmul(tv[0], pv[0]), dmul(tv[1], pv[1])), dmul(tv[2], pv[2])), inv);
  if (u < 0.0 || u > 1.0) return 0;
  qv[0] = dsub(dmul(tv[1], e1[2]), dmul(tv[2], e1[1]));
  qv[1] = dsub(dmul(tv[2], e1[0]), dmul(tv[0], e1[2]));
  qv[2] = dsub(dmul(tv[0], e1[1]), dmul(tv[1], e1[0]));
  const double w = dmul(dadd(dadd(dmul(R[0], qv[0]), dmul(R[1], qv[1])), dmul(R[2], qv[2])), inv);
  if (w < 0.0 || dadd(u, w) > 1.0) return 0;
  const double t = dmul(dadd(dadd(dmul(e2[0], qv[0]), dmul(e2[1], qv[1])), dmul(e2[2], qv[2])), inv);
  return t > 0.0;
}

__device__ int ray_hits_segment(const double* o, const double* p, const double* q) {
  const double dx = dsub(q[0], p[0]), dy = dsub(q[1], p[1]);
  const double den = dsub(dmul(1.0, dy), dmul(kRayY, dx));
  if (den == 0.0) return 0;
  const double px = dsub(p[0], o[0]), py = dsub(p[1], o[1]);
  const double s = __ddiv_rn(dsub(dmul(px, dy), dmul(py, dx)), den);
  const double r = __ddiv_rn(dsub(dmul(px, kRayY), dmul(py, 1.0)), den);
  return s > 0.0 && r >= 0.0 && r < 1.0;
}

__device__ __forceinline__ int lattice_index(const int* m, int v, int ax) {
  return ax == 0 ? v % m[0] : ax == 1 ? (v / m[0]) % m[1] : v / (m[0] * m[1]);
}

__global__ void k_link_check(const DevProblem* __restrict__ probs, const int* __restrict__ cands, int n_cand,
                             int* out) {
  const DevProblem& pr = probs[0];
  const int P = pr.P;
  const long id = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (id >= (long)n_cand * 2 * P) return;
  const int k = (int)(id / (2L * P)), mesh = (int)((id / P) % 2), v = (int)(id % P);
  const double* X = pr.coords + ((size_t)cands[k] * 2 + mesh) * 3 * P;
  const uint8_t fm = pr.fixmask[v];
  const int nfix = (fm & 1) + ((fm >> 1) & 1) + ((fm >> 2) & 1);
  const double o[3] = {X[v], X[P + v], X[2 * (size_t)P + v]};
  int outside = 0;
  if (nfix == 2) {
    const int ax = !(fm & 1) ? 0 : !(fm & 2) ? 1 : 2;
    const int step = ax == 0 ? 1 : ax == 1 ? pr.m[0] : pr.m[0] * pr.m[1];
    const double lo = X[(size_t)ax * P + v - step], hi = X[(size_t)ax * P + v + step];
    outside = !(lo < o[ax] && o[ax] < hi);
  } else if (nfix == 0) {
    int hits = 0;
    for (int s = pr.star_ptr[v]; s < pr.star_ptr[v + 1]; ++s) {
      const int4 tv = pr.tet[pr.star[s]];
      const int ids[4] = {tv.x, tv.y, tv.z, tv.w};
      double V[3][3];
      int n = 0;
      for (int i = 0; i < 4; ++i) {
        if (ids[i] == v) continue;
        for (int a = 0; a < 3; ++a) V[n][a] = X[(size_t)a * P + ids[i]];
        ++n;
      }
      hits += ray_hits_triangle(o, V[0], V[1], V[2]);
    }
    outside = !(hits & 1);
  } else if (nfix == 1) {
    const int f = (fm & 1) ? 0 : (fm & 2) ? 1 : 2;
    const int a1 = f == 0 ? 1 : 0, a2 = f == 2 ? 1 : 2;
    const int fv = lattice_index(pr.m, v, f);
    const double o2[2] = {o[a1], o[a2]};
    int hits = 0;
    for (int s = pr.star_ptr[v]; s < pr.star_ptr[v + 1]; ++s) {
      const int4 tv = pr.tet[pr.star[s]];
      const int ids4[4] = {tv.x, tv.y, tv.z, tv.w};
      int ids[2] = {0, 0}, n = 0;
      for (int i = 0; i < 4; ++i) {
        if (ids4[i] == v) continue;
        if (lattice_index(pr.m, ids4[i], f) == fv) {
          if (n < 2) ids[n] = ids4[i];
          ++n;
        }
      }
      if (n != 2) continue;
      const double p[2] = {X[(size_t)a1 * P + ids[0]], X[(size_t)a2 * P + ids[0]]};
      const double q[2] = {X[(size_t)a1 * P + ids[1]], X[(size_t)a2 * P + ids[1]]};
      hits += ray_hits_segment(o2, p, q);
    }
    outside = !(hits & 1);
  }
  if (outside) atomicAdd(out + 2 * k + mesh, 1);
}

void launch_link_check(const DevProblem* probs, const DevProblem& hp, const int* cands, int n_cand, int* out,
                       cudaStream_t st) {
  const long n = (long)n_cand * 2 * hp.P;
  if (n <= 0) return;
  k_link_check<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(probs, cands, n_cand, out);
}

// Plan deltas from the caller's per-problem [n_groups][n_cand][2][3][G_q]
// arrays into the plan's trial order [slot][2][3][G] (zero beyond G_q).
__global__ void k_gather_deltas(const double* const* raw, const int* slot_q, const long long* slot_src,
                                const int* raw_G, int n_slots, int G, double* out) {
  const long id = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (id >= (long)n_slots * 6 * G) return;
  const long k = id / (6 * G);
  const int r = (int)(id % (6 * G)), ma = r / G, j = r % G;
  const int q = slot_q[k], Gq = raw_G[q];
  out[id] = j < Gq ? raw[q][slot_src[k] + (long)ma * Gq + j] : 0.0;
}

void launch_gather_deltas(const double* const* raw, const int* slot_q, const long long* slot_src, const int* raw_G,
                          int n_slots, int G, double* out, cudaStream_t st) {
  const long n = (long)n_slots * 6 * G;
  if (n <= 0) return;
  k_gather_deltas<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(raw, slot_q, slot_src, raw_G, n_slots, G, out);
}

void launch_setup(const DevProblem* probs, const Batch& b, cudaStream_t st) {
  if (b.n_tt <= 0) return;
  k_setup<<<(unsigned)((2L * b.n_tt + 127) / 128), 128, 0, st>>>(probs, b);
}

// ------------------------------------------------------------ raster + sample
void launch_raster(const DevProblem* probs, const Batch& b, int st_dtype, int warps, int vpw, int n_sm,
                   cudaStream_t st, cudaStream_t side, cudaEvent_t fork) {
  if (b.n_tt <= 0) {
    if (side && fork) {
      cudaEventRecord(fork, st);
      cudaStreamWaitEvent(side, fork, 0);
    }
    return;
  }
  if (st_dtype == ST_F32) launch_raster_f32(probs, b, warps, vpw, n_sm, st, side, fork);
  else if (st_dtype == ST_BF16) launch_raster_bf16(probs, b, warps, vpw, n_sm, st, side, fork);
  else launch_raster_f16(probs, b, warps, vpw, n_sm, st, side, fork);
}

// ------------------------------------------------------------ landmarks
// FP32-filtered inside test of point p (FP64) against the record's tet,
// exact where the margin cannot decide.
__device__ __forceinline__ bool rec_inside(const ItemRec& r, uint32_t fp, const double p[3], float pmag) {
  float px = (float)p[0] - (float)r.O[0], py = (float)p[1] - (float)r.O[1], pz = (float)p[2] - (float)r.O[2];
  unsigned unc = 0;
  for (int f = 0; f < 4; ++f) {
    float h = fmaf(r.fa[f][0], px, fmaf(r.fa[f][1], py, fmaf(r.fa[f][2], pz, r.fa[f][3])));
    float an = fabsf(r.fa[f][0]) + fabsf(r.fa[f][1]) + fabsf(r.fa[f][2]);
    float qm = fmaxf(fabsf(px), fmaxf(fabsf(py), fabsf(pz)));
    float mu = r.fm[f][0] + r.fm[f][2] * qm + an * (pmag + fabsf(px) + fabsf(py) + fabsf(pz) + 1.0f) * (1.0f / 1048576.0f);
    if (h < -mu) return false;
    if (!(h > mu)) unc |= 1u << f;
  }
  for (int f = 0; f < 4; ++f)
    if ((unc >> f) & 1)
      if (!rec_face_in_exact(r, fp, f, p)) return false;
  return true;
}

// Faces of records are only filled for tets with positive own volume and a
// non-empty clipped box; a landmark test needs the faces even when the box
// is empty, so the landmark kernels treat "no faces" conservatively by the
// exact predicate.
__device__ __noinline__ bool rec_inside_exact_all(const ItemRec& r, uint32_t fp, const double p[3]) {
  for (int f = 0; f < 4; ++f)
    if (!rec_face_in_exact(r, fp, f, p)) return false;
  return true;
}

__device__ __forceinline__ bool vol_positive(const ItemRec& r) {
  // the record keeps the own vertices; recompute 6V exactly
  double e[3][3], r1[3];
  for (int i = 0; i < 3; ++i)
    for (int a = 0; a < 3; ++a) e[i][a] = dsub(r.X[i + 1][a], r.X[0][a]);
  cross3d(e[1], e[2], r1);
  double v = dot3d(e[0], r1);
  return v > 0 && isfinite(v);
}

// Sec. 2.3.3: smallest squared physical distance between guidance point i
// of mesh `mesh` (at p), mapped through the record's tet, and the partner
// points of its set (its own partner when there are no sets).  The mapped
// point is p + disp with disp = d0 + G (p - own_0) small, so the distance
// vector (p - q) + disp is formed from the FP64 differences p - own_0,
// d0 and p - q rounded once to FP32 and the FP32 map: a few 1e-7 of the
// distance, with a dozen FP64 operations instead of ~40 (this runs on one
// lane, and an FP64 instruction occupies the pipe for the whole warp).
__device__ double landmark_term(const ItemRec& r, const DevProblem& pr, const double p[3], int mesh, int i) {
  float u[3], disp[3];
  for (int a = 0; a < 3; ++a) u[a] = (float)dsub(p[a], r.X[0][a]);
  for (int c = 0; c < 3; ++c)
    disp[c] = (float)dsub(r.XP[0][c], r.X[0][c]) + fmaf(r.G[c][0], u[0], fmaf(r.G[c][1], u[1], r.G[c][2] * u[2]));
  const int dp = 1 - mesh;
  int k0 = 0, k1 = 1;
  if (pr.gsid) {
    const int s = pr.gsid[i];
    k0 = pr.gptr[s];
    k1 = pr.gptr[s + 1];
  }
  float best = INFINITY;
  for (int k = k0; k < k1; ++k) {
    const int j = pr.gsid ? pr.gmem[k] : i;
    const double* q = pr.guide + 6 * j + 3 * (1 - mesh);
    float t = 0.f;
    for (int a = 0; a < 3; ++a) {
      const float d = ((float)dsub(p[a], q[a]) + disp[a]) * pr.sp[dp][a];
      t = fmaf(d, d, t);
    }
    best = t < best ? t : best;
  }
  return (double)best;
}

// Test one tet record for landmark p: volume sign first (folded tets never
// contain a point), then the filtered face tests.
__device__ __forceinline__ bool lm_test(const ItemRec& r, uint32_t fp, const double p[3], float pmag) {
  if (r.flags & 1) return rec_inside(r, fp, p, pmag);
  if (!vol_positive(r)) return false;
  return rec_inside_exact_all(r, fp, p);
}

// Full evaluation: one warp per (candidate, mesh, landmark) scans all tets
// in index order (Sec. 2.3.3).
__global__ void k_locate_full(const DevProblem* probs, Batch b, int c0, int nc) {
  const DevProblem& pr = probs[0];
  int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  int ng = pr.ng;
  if (gw >= nc * 2 * ng) return;
  int ci = gw / (2 * ng);
  int rem = gw % (2 * ng);
  int mesh = rem / ng, i = rem % ng;
  int cand = c0 + ci;
  double p[3];
  for (int a = 0; a < 3; ++a) p[a] = pr.guide[6 * i + 3 * mesh + a];
  float pmag = fmaxf(fabsf((float)p[0]), fmaxf(fabsf((float)p[1]), fabsf((float)p[2])));
  int found = -1;
  for (int tb = 0; tb < pr.ntet && found < 0; tb += 32) {
    int t = tb + lane;
    bool in = false;
    if (t < pr.ntet) {
      const ItemRec& r = b.rec[2 * ((size_t)ci * pr.ntet + t) + mesh];
      in = lm_test(r, pr.fperm[t], p, pmag);
    }
    unsigned m = __ballot_sync(FULL_MASK, in);
    if (m) found = tb + __ffs(m) - 1;
  }
  if (lane == 0) {
    size_t li = ((size_t)cand * 2 + mesh) * ng + i;
    pr.c_loc[li] = found;
    pr.c_gterm[li] = found >= 0 ? landmark_term(b.rec[2 * ((size_t)ci * pr.ntet + found) + mesh], pr, p, mesh, i) : 0.0;
  }
}

void launch_locate_full(const DevProblem* probs, const DevProblem& hp, const Batch& b, int c0, int nc,
                        cudaStream_t st) {
  long warps = (long)nc * 2 * hp.ng;
  if (warps <= 0) return;
  k_locate_full<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(probs, b, c0, nc);
}

// Full evaluation: ordered FP64 sums per candidate (tets, then landmarks).
__global__ void k_reduce_full(const DevProblem* probs, int c0, int nc, double* obj) {
  const DevProblem& pr = probs[0];
  int ci = blockIdx.x * blockDim.x + threadIdx.x;
  if (ci >= nc) return;
  int c = c0 + ci;
  double raw[4] = {0, 0, 0, 0};
  unsigned long long cov = 0;
  for (int t = 0; t < pr.ntet; ++t) {
    size_t j = (size_t)c * pr.ntet + t;
    raw[0] = dadd(raw[0], dadd(pr.c_ssd[2 * j], pr.c_ssd[2 * j + 1]));
    raw[1] = dadd(raw[1], pr.c_def[j]);
    raw[3] = dadd(raw[3], (double)pr.c_fold[j]);
    cov += (unsigned)(pr.c_cov[2 * j] + pr.c_cov[2 * j + 1]);
  }
  for (int mesh = 0; mesh < 2; ++mesh)
    for (int i = 0; i < pr.ng; ++i) {
      size_t li = ((size_t)c * 2 + mesh) * pr.ng + i;
      if (pr.c_loc[li] < 0) raw[3] = dadd(raw[3], 1.0);
      raw[2] = dadd(raw[2], pr.c_gterm[li]);
    }
  for (int q = 0; q < 4; ++q) pr.sums[4 * (size_t)c + q] = raw[q];
  if (obj) {
    obj[4 * (size_t)ci + 0] = raw[0] / pr.sim_norm;
    obj[4 * (size_t)ci + 1] = raw[1] / pr.def_norm;
    obj[4 * (size_t)ci + 2] = pr.ng > 0 ? raw[2] / pr.guid_norm : 0.0;
    obj[4 * (size_t)ci + 3] = raw[3];
  }
  atomicAdd(pr.samples, cov);
}

void launch_reduce_full(const DevProblem* probs, int c0, int nc, const Batch& b, double* obj, cudaStream_t st) {
  (void)b;
  k_reduce_full<<<(nc + 127) / 128, 128, 0, st>>>(probs, c0, nc, obj);
}

// Partial evaluation: one warp per trial relocates the landmarks whose
// current tet is touched (or that are unlocated) among the touched tets.
// The trial's sorted touched-tet list is staged in shared memory so the
// membership searches do not chain global loads.
constexpr int kLmWarps = 8;
constexpr int kLmTl = 256;  // staged list length per warp; longer lists search global memory

__device__ __forceinline__ bool sorted_has(const int* tl, int n, int v) {
  int lo = 0, hi = n - 1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    int x = tl[mid];
    if (x == v) return true;
    if (x < v) lo = mid + 1;
    else hi = mid - 1;
  }
  return false;
}

// Partial evaluation, guidance points (Sec. 2.3.3): one warp per trial.  The
// points whose cached tet the trial touches (or that are unlocated) are taken
// 32 at a time in index order: the lanes first test all (point, touched tet)
// pairs (the lowest tet index that contains a point wins, as a scan in order
// would find), then evaluate the points' terms side by side; the changes are
// added on one lane in index order.
__global__ void __launch_bounds__(32 * kLmWarps, 3) k_landmarks_partial(const DevProblem* probs, Batch b) {
  __shared__ int s_tl[kLmWarps][kLmTl];
  __shared__ int s_found[kLmWarps][32];
  __shared__ double s_dg[kLmWarps][32];
  const int w = threadIdx.x >> 5;
  int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (k >= b.n_trials) return;
  const DevProblem& pr = probs[b.tr_prob ? b.tr_prob[k] : 0];
  const int ng = pr.ng;
  const int cand = b.tr_cand[k];
  const int first = b.tr_first[k], ntt = b.tr_ntt[k];
  const int* tl = b.tt_tet + first;
  int* stl = s_tl[w];
  const bool staged = ntt <= kLmTl;
  if (staged)
    for (int j = lane; j < ntt; j += 32) stl[j] = tl[j];
  __syncwarp();
  const int* sl = staged ? stl : tl;
  int naff = 0;
  double gd = 0.0;
  int ud = 0;
  for (int base = 0; base < 2 * ng; base += 32) {
    const int e = base + lane;
    bool aff = false;
    int told = -2;
    if (e < 2 * ng) {
      const int mesh = e / ng, i = e % ng;
      told = pr.c_loc[((size_t)cand * 2 + mesh) * ng + i];
      aff = told < 0 || sorted_has(sl, ntt, told);
    }
    const unsigned am = __ballot_sync(FULL_MASK, aff);
    if (!am) continue;
    const int na = __popc(am);
    // slot of this lane's point among the affected ones, in index order
    const int slot = __popc(am & ((1u << lane) - 1u));
    s_found[w][lane] = INT_MAX;
    __syncwarp();
    // (affected point, touched tet) pairs
    for (int q = lane; q < na * ntt; q += 32) {
      const int a = q / ntt, j = q - a * ntt;
      const int src = __fns(am, 0, a + 1);  // lane of the a-th affected point
      const int ee = base + src;
      const int mesh = ee / ng, i = ee % ng;
      double pp[3];
      for (int c = 0; c < 3; ++c) pp[c] = pr.guide[6 * i + 3 * mesh + c];
      const float pmag = fmaxf(fabsf((float)pp[0]), fmaxf(fabsf((float)pp[1]), fabsf((float)pp[2])));
      const ItemRec& r = b.rec[2 * (size_t)(first + j) + mesh];
      if (lm_test(r, pr.fperm[sl[j]], pp, pmag)) atomicMin(&s_found[w][a], j);
    }
    __syncwarp();
    if (aff) {
      const int mesh = e / ng, i = e % ng;
      double pp[3];
      for (int c = 0; c < 3; ++c) pp[c] = pr.guide[6 * i + 3 * mesh + c];
      const int fj = s_found[w][slot];
      const int found = fj == INT_MAX ? -1 : fj;
      const double term = found >= 0 ? landmark_term(b.rec[2 * (size_t)(first + found) + mesh], pr, pp, mesh, i) : 0.0;
      const size_t li = ((size_t)cand * 2 + mesh) * ng + i;
      s_dg[w][slot] = dsub(term, pr.c_gterm[li]);
      if (naff + slot < b.aff_cap) {
        const size_t o = (size_t)k * b.aff_cap + naff + slot;
        b.aff_idx[o] = e;
        b.aff_loc[o] = found >= 0 ? sl[found] : -1;
        b.aff_term[o] = term;
      }
      ud += (found < 0 ? 1 : 0) - (told < 0 ? 1 : 0);
    }
    __syncwarp();
    if (lane == 0)
      for (int a = 0; a < na; ++a) gd = dadd(gd, s_dg[w][a]);
    naff += na;
  }
  ud = __reduce_add_sync(FULL_MASK, ud);
  if (lane == 0) {
    b.aff_n[k] = min(naff, b.aff_cap);
    b.tr_delta[4 * (size_t)k + 2] = gd;
    b.tr_delta[4 * (size_t)k + 3] = (double)ud;
  }
}

void launch_landmarks_partial(const DevProblem* probs, const Batch& b, cudaStream_t st) {
  if (b.n_trials <= 0) return;
  long threads = 32L * b.n_trials;
  k_landmarks_partial<<<(unsigned)((threads + 32 * kLmWarps - 1) / (32 * kLmWarps)), 32 * kLmWarps, 0, st>>>(probs, b);
}

// Partial evaluation: new = stored - sum old + sum new over touched tets.
// One warp per trial: lanes take the touched tets, FP64 warp sums.
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = dadd(v, __shfl_xor_sync(FULL_MASK, v, o));
  return v;
}

// Trial k's deltas (one warp; lane 0 writes tr_delta and, with write_obj,
// tr_obj); returns the trial's sample count on every lane.  GB300 issues an
// FP64 instruction at a small fraction of the FP32 rate whatever the number
// of active lanes, so the sums are arranged for few FP64 instructions: each
// lane adds the per-tet differences new - old of its tets, the fold counts
// are integers, and the two FP64 sums share one butterfly (lanes 0-15 carry
// the dissimilarity, lanes 16-31 the deformation after the first exchange).
__device__ __forceinline__ unsigned reduce_trial(const DevProblem& pr, const Batch& b, int k, int lane,
                                                 int has_landmarks, bool write_obj) {
  const int cand = b.tr_cand[k];
  const int first = b.tr_first[k], ntt = b.tr_ntt[k];
  double ds = 0.0, dd = 0.0;
  int dfold = 0;
  unsigned cov = 0;
  for (int j = lane; j < ntt; j += 32) {
    const int tt = first + j;
    const size_t ci = (size_t)cand * pr.ntet + b.tt_tet[tt];
    ds = dadd(ds, dsub(dadd(b.o_ssd[2 * (size_t)tt], b.o_ssd[2 * (size_t)tt + 1]),
                       dadd(pr.c_ssd[2 * ci], pr.c_ssd[2 * ci + 1])));
    dd = dadd(dd, dsub(b.o_def[tt], pr.c_def[ci]));
    dfold += b.o_fold[tt] - pr.c_fold[ci];
    cov += (unsigned)(b.o_cov[2 * (size_t)tt] + b.o_cov[2 * (size_t)tt + 1]);
  }
  const bool upper = lane >= 16;
  double v = upper ? dd : ds;
  v = dadd(v, __shfl_xor_sync(FULL_MASK, upper ? ds : dd, 16));
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v = dadd(v, __shfl_xor_sync(FULL_MASK, v, o));
  const double sum_dd = __shfl_sync(FULL_MASK, v, 16);
  dfold = __reduce_add_sync(FULL_MASK, dfold);
  cov = __reduce_add_sync(FULL_MASK, cov);
  if (lane == 0) {
    double* dl = b.tr_delta + 4 * (size_t)k;
    dl[0] = v;
    dl[1] = sum_dd;
    const double gd = has_landmarks ? dl[2] : 0.0;
    const double ud = has_landmarks ? dl[3] : 0.0;
    if (!has_landmarks) dl[2] = 0.0;
    dl[3] = dadd((double)dfold, ud);
    if (write_obj) {
      const double* s = pr.sums + 4 * (size_t)cand;
      double* ob = b.tr_obj + 4 * (size_t)k;
      ob[0] = dadd(s[0], dl[0]) / pr.sim_norm;
      ob[1] = dadd(s[1], dl[1]) / pr.def_norm;
      ob[2] = pr.ng > 0 ? dadd(s[2], gd) / pr.guid_norm : 0.0;
      ob[3] = dadd(s[3], dl[3]);
    }
  }
  return cov;
}

__global__ void k_reduce_partial(const DevProblem* probs, Batch b, int has_landmarks) {
  int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (k >= b.n_trials) return;
  const DevProblem& pr = probs[b.tr_prob ? b.tr_prob[k] : 0];
  const unsigned cov = reduce_trial(pr, b, k, lane, has_landmarks, true);
  if (lane == 0) atomicAdd(pr.samples, (unsigned long long)cov);
}

void launch_reduce_partial(const DevProblem* probs, const Batch& b, cudaStream_t st) {
  if (b.n_trials <= 0) return;
  long threads = 32L * b.n_trials;
  k_reduce_partial<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(probs, b, b.aff_n != nullptr);
}

// Accept-if-improves (Sec. 2.2), constraint domination first.
// The objectives are the raw sums over positive constants, so the trial is
// compared with the candidate in sums (after the deltas of reduce_trial):
// constraint domination first, then weak Pareto dominance with one strict
// improvement.
__device__ __forceinline__ bool accept_trial(const DevProblem& pr, const Batch& b, int k) {
  const double* s = pr.sums + 4 * (size_t)b.tr_cand[k];
  const double* dl = b.tr_delta + 4 * (size_t)k;
  const double n3 = dadd(s[3], dl[3]);
  if (n3 != s[3]) return n3 < s[3];
  const double n0 = dadd(s[0], dl[0]), n1 = dadd(s[1], dl[1]);
  const double n2 = pr.ng > 0 ? dadd(s[2], dl[2]) : s[2];
  const bool le = n0 <= s[0] && n1 <= s[1] && n2 <= s[2];
  const bool lt = n0 < s[0] || n1 < s[1] || n2 < s[2];
  return le && lt;
}

__global__ void k_accept(const DevProblem* probs, Batch b, uint8_t* accept) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= b.n_trials) return;
  const DevProblem& pr = probs[b.tr_prob ? b.tr_prob[k] : 0];
  accept[k] = accept_trial(pr, b, k) ? 1 : 0;
}

void launch_accept(const DevProblem* probs, const Batch& b, uint8_t* accept, cudaStream_t st) {
  if (b.n_trials <= 0) return;
  k_accept<<<(b.n_trials + 127) / 128, 128, 0, st>>>(probs, b, accept);
}

// Commit: per touched tet (cache), per trial (coords, landmarks), per
// candidate (sum of the accepted deltas).
__global__ void k_commit_tt(const DevProblem* probs, Batch b, const uint8_t* accept) {
  int tt = blockIdx.x * blockDim.x + threadIdx.x;
  if (tt >= b.n_tt) return;
  int k = b.tt_trial[tt];
  if (!accept[k]) return;
  const DevProblem& pr = probs[b.tr_prob ? b.tr_prob[k] : 0];
  size_t ci = (size_t)b.tr_cand[k] * pr.ntet + b.tt_tet[tt];
  pr.c_ssd[2 * ci] = b.o_ssd[2 * (size_t)tt];
  pr.c_ssd[2 * ci + 1] = b.o_ssd[2 * (size_t)tt + 1];
  pr.c_cov[2 * ci] = b.o_cov[2 * (size_t)tt];
  pr.c_cov[2 * ci + 1] = b.o_cov[2 * (size_t)tt + 1];
  pr.c_def[ci] = b.o_def[tt];
  pr.c_fold[ci] = b.o_fold[tt];
}

__global__ void k_commit_trial(const DevProblem* probs, Batch b, const uint8_t* accept, const int* tr_group,
                               const int* g_ptr, const int* g_pts) {
  int k = blockIdx.x;
  if (k >= b.n_trials || !accept[k]) return;
  const DevProblem& pr = probs[b.tr_prob ? b.tr_prob[k] : 0];
  const int cand = b.tr_cand[k];
  const int g = tr_group[k];
  const int np = g_ptr[g + 1] - g_ptr[g];
  for (int e = threadIdx.x; e < 6 * np; e += blockDim.x) {
    int ma = e / np, j = e % np;
    int pid = g_pts[g_ptr[g] + j];
    pr.coords[((size_t)cand * 6 + ma) * pr.P + pid] = b.tr_coords[(size_t)k * 6 * b.gmax + (size_t)ma * b.gmax + j];
  }
  if (b.aff_n) {
    int na = b.aff_n[k];
    for (int e = threadIdx.x; e < na; e += blockDim.x) {
      size_t o = (size_t)k * b.aff_cap + e;
      int idx = b.aff_idx[o];
      size_t li = (size_t)cand * 2 * pr.ng + idx;
      pr.c_loc[li] = b.aff_loc[o];
      pr.c_gterm[li] = b.aff_term[o];
    }
  }
}

// One warp per candidate: the accepted trials' deltas (independent groups)
// summed over the warp, then added to the stored sums.
__global__ void k_commit_sums(const DevProblem* probs, Batch b, const uint8_t* accept, const int* cand_ptr,
                              const int* cand_trials, int n_list) {
  int ci = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (ci >= n_list) return;
  const int j0 = cand_ptr[ci], j1 = cand_ptr[ci + 1];
  if (j1 <= j0) return;
  int k0 = cand_trials[j0];
  const DevProblem& pr = probs[b.tr_prob ? b.tr_prob[k0] : 0];
  // each lane adds its accepted trials' deltas, then one butterfly carries
  // all four sums (lanes 0-7, 8-15, 16-23, 24-31 end with delta 0, 1, 2, 3):
  // few FP64 instructions
  double d[4] = {0, 0, 0, 0};
  for (int j = j0 + lane; j < j1; j += 32) {
    const int k = cand_trials[j];
    if (accept[k])
      for (int q = 0; q < 4; ++q) d[q] = dadd(d[q], b.tr_delta[4 * (size_t)k + q]);
  }
  const bool up16 = (lane & 16) != 0, up8 = (lane & 8) != 0;
  const double a0 = dadd(up16 ? d[2] : d[0], __shfl_xor_sync(FULL_MASK, up16 ? d[0] : d[2], 16));
  const double a1 = dadd(up16 ? d[3] : d[1], __shfl_xor_sync(FULL_MASK, up16 ? d[1] : d[3], 16));
  double v = dadd(up8 ? a1 : a0, __shfl_xor_sync(FULL_MASK, up8 ? a0 : a1, 8));
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) v = dadd(v, __shfl_xor_sync(FULL_MASK, v, o));
  double tot[4];
  tot[0] = __shfl_sync(FULL_MASK, v, 0);
  tot[1] = __shfl_sync(FULL_MASK, v, 8);
  tot[2] = __shfl_sync(FULL_MASK, v, 16);
  tot[3] = __shfl_sync(FULL_MASK, v, 24);
  if (lane == 0) {
    double* s = pr.sums + 4 * (size_t)b.tr_cand[k0];
    for (int q = 0; q < 4; ++q) s[q] = dadd(s[q], tot[q]);
  }
}

// Generation plans: reduce, accept and the per-trial part of the commit in
// one warp per trial.  The trials of a wave touch disjoint tets and move
// disjoint points, and every accept decision reads the candidate's sums
// from before the wave (k_commit_sums, launched after, adds the accepted
// deltas), so committing a trial's tets, coordinates and guidance points
// right after its decision gives the same state as the separate kernels.
// Sample counts are added once per block.
__global__ void __launch_bounds__(256) k_reduce_commit(const DevProblem* probs, Batch b, int has_landmarks,
                                                       uint8_t* accept, const int* tr_group, const int* g_ptr,
                                                       const int* g_pts) {
  __shared__ unsigned long long s_cov[8];
  __shared__ int s_pi[8];
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int pi = (k < b.n_trials && b.tr_prob) ? b.tr_prob[k] : 0;
  const DevProblem& pr = probs[pi];
  unsigned cov = 0;
  if (k < b.n_trials) {
    cov = reduce_trial(pr, b, k, lane, has_landmarks, false);
    int acc = 0;
    if (lane == 0) {
      acc = accept_trial(pr, b, k) ? 1 : 0;
      accept[k] = (uint8_t)acc;
    }
    acc = __shfl_sync(FULL_MASK, acc, 0);
    if (acc) {
      const int cand = b.tr_cand[k];
      const int first = b.tr_first[k], ntt = b.tr_ntt[k];
      for (int j = lane; j < ntt; j += 32) {
        const int tt = first + j;
        const size_t ci = (size_t)cand * pr.ntet + b.tt_tet[tt];
        pr.c_ssd[2 * ci] = b.o_ssd[2 * (size_t)tt];
        pr.c_ssd[2 * ci + 1] = b.o_ssd[2 * (size_t)tt + 1];
        pr.c_cov[2 * ci] = b.o_cov[2 * (size_t)tt];
        pr.c_cov[2 * ci + 1] = b.o_cov[2 * (size_t)tt + 1];
        pr.c_def[ci] = b.o_def[tt];
        pr.c_fold[ci] = b.o_fold[tt];
      }
      const int g = tr_group[k];
      const int np = g_ptr[g + 1] - g_ptr[g];
      for (int e = lane; e < 6 * np; e += 32) {
        const int ma = e / np, j = e % np;
        const int pid = g_pts[g_ptr[g] + j];
        pr.coords[((size_t)cand * 6 + ma) * pr.P + pid] = b.tr_coords[(size_t)k * 6 * b.gmax + (size_t)ma * b.gmax + j];
      }
      if (b.aff_n) {
        const int na = b.aff_n[k];
        for (int e = lane; e < na; e += 32) {
          const size_t o = (size_t)k * b.aff_cap + e;
          const size_t li = (size_t)cand * 2 * pr.ng + b.aff_idx[o];
          pr.c_loc[li] = b.aff_loc[o];
          pr.c_gterm[li] = b.aff_term[o];
        }
      }
    }
  }
  if (lane == 0) {
    s_cov[w] = cov;
    s_pi[w] = pi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // one atomic per run of warps of the same problem
    unsigned long long t = 0;
    const int nw = (int)(blockDim.x >> 5);
    for (int i = 0; i < nw; ++i) {
      t += s_cov[i];
      if (i + 1 == nw || s_pi[i + 1] != s_pi[i]) {
        if (t) atomicAdd(probs[s_pi[i]].samples, t);
        t = 0;
      }
    }
  }
}

void launch_reduce_commit(const DevProblem* probs, const Batch& b, uint8_t* accept, const int* tr_group,
                          const int* g_ptr, const int* g_pts, const int* cand_ptr, const int* cand_trials, int n_list,
                          cudaStream_t st, cudaStream_t sums_st, cudaEvent_t sums_ev) {
  if (b.n_trials <= 0) return;
  const long threads = 32L * b.n_trials;
  k_reduce_commit<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(probs, b, b.aff_n != nullptr, accept, tr_group,
                                                                      g_ptr, g_pts);
  cudaStream_t ss = st;
  if (sums_st && sums_ev) {
    cudaEventRecord(sums_ev, st);
    cudaStreamWaitEvent(sums_st, sums_ev, 0);
    ss = sums_st;
  }
  k_commit_sums<<<(unsigned)((32L * n_list + 255) / 256), 256, 0, ss>>>(probs, b, accept, cand_ptr, cand_trials, n_list);
}

void launch_commit(const DevProblem* probs, const Batch& b, const uint8_t* accept, const int* tr_group,
                   const int* g_ptr, const int* g_pts, const int* cand_ptr, const int* cand_trials, int n_list,
                   cudaStream_t st) {
  if (b.n_trials <= 0) return;
  k_commit_tt<<<(b.n_tt + 255) / 256, 256, 0, st>>>(probs, b, accept);
  k_commit_trial<<<b.n_trials, 64, 0, st>>>(probs, b, accept, tr_group, g_ptr, g_pts);
  k_commit_sums<<<(unsigned)((32L * n_list + 255) / 256), 256, 0, st>>>(probs, b, accept, cand_ptr, cand_trials, n_list);
}

// Proposal for generation plans: trial coords = committed group coords + delta.
__global__ void k_propose(const DevProblem* probs, Batch b, const int* tr_group, const int* g_ptr, const int* g_pts,
                          const double* deltas) {
  int k = blockIdx.x;
  if (k >= b.n_trials) return;
  const DevProblem& pr = probs[b.tr_prob ? b.tr_prob[k] : 0];
  const int cand = b.tr_cand[k];
  const int g = tr_group[k];
  const int np = g_ptr[g + 1] - g_ptr[g];
  double* out = (double*)b.tr_coords + (size_t)k * 6 * b.gmax;
  const double* dl = deltas + (size_t)k * 6 * b.gmax;
  for (int e = threadIdx.x; e < 6 * np; e += blockDim.x) {
    int ma = e / np, j = e % np;
    int pid = g_pts[g_ptr[g] + j];
    out[(size_t)ma * b.gmax + j] = pr.coords[((size_t)cand * 6 + ma) * pr.P + pid] + dl[(size_t)ma * b.gmax + j];
  }
}

void launch_propose(const DevProblem* probs, const Batch& b, const int* tr_group, const int* g_ptr, const int* g_pts,
                    const double* deltas, cudaStream_t st) {
  if (b.n_trials <= 0) return;
  k_propose<<<b.n_trials, 64, 0, st>>>(probs, b, tr_group, g_ptr, g_pts, deltas);
}

}  // namespace dmr
