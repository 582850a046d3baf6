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

namespace dmr {

#define FULL_MASK 0xffffffffu

// ------------------------------------------------------------ FP64 exact
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }

__device__ __forceinline__ void cross3d(const double a[3], const double b[3], double o[3]) {
  o[0] = dsub(dmul(a[1], b[2]), dmul(a[2], b[1]));
  o[1] = dsub(dmul(a[2], b[0]), dmul(a[0], b[2]));
  o[2] = dsub(dmul(a[0], b[1]), dmul(a[1], b[0]));
}
__device__ __forceinline__ double dot3d(const double a[3], const double b[3]) {
  return dadd(dmul(a[0], b[0]), dadd(dmul(a[1], b[1]), dmul(a[2], b[2])));
}

// Exact face predicate: canonical face (a,b,c) with inward sign s; p on the
// inner side, or on the plane and the signed normal's first nonzero
// component in (z, y, x) order is positive.
__device__ __noinline__ bool face_in_exact(const double* A, const double* B, const double* Cc, int s,
                                           const double p[3]) {
  double u[3], w[3], n[3];
  for (int k = 0; k < 3; ++k) {
    u[k] = dsub(B[k], A[k]);
    w[k] = dsub(Cc[k], A[k]);
  }
  cross3d(u, w, n);
  double g = dadd(dmul(n[0], dsub(p[0], A[0])), dadd(dmul(n[1], dsub(p[1], A[1])), dmul(n[2], dsub(p[2], A[2]))));
  double h = s > 0 ? g : -g;
  if (h > 0) return true;
  if (h == 0) {
    double mz = s > 0 ? n[2] : -n[2];
    double my = s > 0 ? n[1] : -n[1];
    double mx = s > 0 ? n[0] : -n[0];
    if (mz != 0) return mz > 0;
    if (my != 0) return my > 0;
    return mx > 0;
  }
  return false;
}

__device__ __forceinline__ int face_local(uint32_t fp, int f, int which) { return (fp >> (8 * f + 2 * which)) & 3; }
__device__ __forceinline__ int face_sign(uint32_t fp, int f) { return ((fp >> (8 * f + 6)) & 1) ? -1 : 1; }

// Exact face test of face f of the record's own tet at point p.
__device__ __forceinline__ bool rec_face_in_exact(const ItemRec& r, uint32_t fp, int f, const double p[3]) {
  int ia = face_local(fp, f, 0), ib = face_local(fp, f, 1), ic = face_local(fp, f, 2);
  return face_in_exact(r.X[ia], r.X[ib], r.X[ic], face_sign(fp, f), p);
}

// FP64 mapped coordinate, the definition the black decision follows:
// p' = (v + d0) + G (v - own_0).
__device__ __noinline__ void map_exact(const ItemRec& r, const double v[3], double out[3]) {
  double q[3];
  for (int a = 0; a < 3; ++a) q[a] = dsub(v[a], r.X[0][a]);
  for (int c = 0; c < 3; ++c)
    out[c] = dadd(dadd(v[c], r.d0[c]),
                  dadd(dmul(r.G64[c][0], q[0]), dadd(dmul(r.G64[c][1], q[1]), dmul(r.G64[c][2], q[2]))));
}

// ------------------------------------------------------------ float helpers
#define MAGIC 12582912.0f /* 1.5 * 2^23 */
#define MAGIC_BITS 0x4B400000

// floor for |x| < 2^22 with two full-rate ALU ops: returns the float floor
// and the integer floor + MAGIC_BITS (as raw bits).
__device__ __forceinline__ float ffloor_magic(float x, int& ibits) {
  float t = __fadd_rd(x, MAGIC);
  ibits = __float_as_int(t);
  return t - MAGIC;
}

__device__ __forceinline__ float bf16lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
__device__ __forceinline__ float f16lo(uint32_t w) { return __half2float(__ushort_as_half((unsigned short)(w & 0xffff))); }
__device__ __forceinline__ float f16hi(uint32_t w) { return __half2float(__ushort_as_half((unsigned short)(w >> 16))); }

template <int ST>
__device__ __forceinline__ float load_plain(const void* p, long i) {
  if (ST == ST_F32) return __ldg((const float*)p + i);
  unsigned short u = __ldg((const unsigned short*)p + i);
  if (ST == ST_BF16) return __uint_as_float((uint32_t)u << 16);
  return __half2float(__ushort_as_half(u));
}

__device__ __forceinline__ float load_plain_dyn(const void* p, int st, long i) {
  if (st == ST_F32) return load_plain<ST_F32>(p, i);
  if (st == ST_BF16) return load_plain<ST_BF16>(p, i);
  return load_plain<ST_F16>(p, i);
}

// Trilinear interpolation of a corner-packed cell: corner index dx+2dy+4dz.
template <int ST>
__device__ __forceinline__ float cell_lerp(const void* cells, unsigned idx, float fx, float fy, float fz) {
  float c0, c1, c2, c3, c4, c5, c6, c7;
  if (ST == ST_F32) {
    const float4* p = (const float4*)cells + 2 * (size_t)idx;
    float4 a = __ldg(p), b = __ldg(p + 1);
    c0 = a.x; c1 = a.y; c2 = a.z; c3 = a.w; c4 = b.x; c5 = b.y; c6 = b.z; c7 = b.w;
  } else {
    uint4 w = __ldg((const uint4*)cells + idx);
    if (ST == ST_BF16) {
      c0 = bf16lo(w.x); c1 = bf16hi(w.x); c2 = bf16lo(w.y); c3 = bf16hi(w.y);
      c4 = bf16lo(w.z); c5 = bf16hi(w.z); c6 = bf16lo(w.w); c7 = bf16hi(w.w);
    } else {
      c0 = f16lo(w.x); c1 = f16hi(w.x); c2 = f16lo(w.y); c3 = f16hi(w.y);
      c4 = f16lo(w.z); c5 = f16hi(w.z); c6 = f16lo(w.w); c7 = f16hi(w.w);
    }
  }
  float a0 = fmaf(fx, c1 - c0, c0);
  float a1 = fmaf(fx, c3 - c2, c2);
  float a2 = fmaf(fx, c5 - c4, c4);
  float a3 = fmaf(fx, c7 - c6, c6);
  float b0 = fmaf(fy, a1 - a0, a0);
  float b1 = fmaf(fy, a3 - a2, a2);
  return fmaf(fz, b1 - b0, b0);
}

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

__global__ void k_build_cells(const void* plain, int st, int nx, int ny, int nz, void* cells, uint8_t* cflag) {
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
  if (st == ST_F32) {
    float4* p = (float4*)cells + 2 * id;
    p[0] = make_float4(fv[0], fv[1], fv[2], fv[3]);
    p[1] = make_float4(fv[4], fv[5], fv[6], fv[7]);
  } else {
    uint4 w;
    w.x = raw[0] | (raw[1] << 16);
    w.y = raw[2] | (raw[3] << 16);
    w.z = raw[4] | (raw[5] << 16);
    w.w = raw[6] | (raw[7] << 16);
    ((uint4*)cells)[id] = w;
  }
  cflag[id] = (uint8_t)(any0 | (all0 << 1));
}

void launch_build_cells(const void* plain, int dtype, const int n[3], void* cells, uint8_t* cflag, cudaStream_t st) {
  long N = (long)(n[0] + 2) * (n[1] + 2) * (n[2] + 2);
  k_build_cells<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(plain, dtype, n[0], n[1], n[2], cells, cflag);
}

// ------------------------------------------------------------ geometry set-up
__device__ __forceinline__ double vcoord(const DevProblem& pr, const Batch& b, int k, int cand, uint32_t slots,
                                         int i, int vid, int mesh, int axis) {
  int sl = (int)((slots >> (8 * i)) & 0xff) - 1;
  if (sl >= 0) return b.tr_coords[(size_t)k * 6 * b.gmax + (size_t)(mesh * 3 + axis) * b.gmax + sl];
  return pr.coords[((size_t)cand * 6 + mesh * 3 + axis) * pr.P + vid];
}

__device__ __forceinline__ float fabs3max(float a, float b, float c) { return fmaxf(fabsf(a), fmaxf(fabsf(b), fabsf(c))); }

// One thread per (trial, tet): fold count, deformation, and the two
// direction records (Sec. 2.3.1-2.3.4).
__global__ void __launch_bounds__(128) k_setup(const DevProblem* probs, Batch b) {
  int tt = blockIdx.x * blockDim.x + threadIdx.x;
  if (tt == 0 && b.work) *b.work = 0u;
  if (tt >= b.n_tt) return;
  int k = b.tt_trial[tt];
  int t = b.tt_tet[tt];
  const int pi = b.tr_prob ? b.tr_prob[k] : 0;
  const DevProblem& pr = probs[pi];
  int cand = b.tr_cand[k];
  int4 tv = pr.tet[t];
  int vid[4] = {tv.x, tv.y, tv.z, tv.w};
  uint32_t slots = b.tt_slot ? b.tt_slot[tt] : 0u;
  double X[2][4][3];
  for (int mesh = 0; mesh < 2; ++mesh)
    for (int i = 0; i < 4; ++i)
      for (int a = 0; a < 3; ++a) X[mesh][i][a] = vcoord(pr, b, k, cand, slots, i, vid[i], mesh, a);

  // edge vectors, differences, fold (FP64, oracle expression order)
  double e[2][3][3];
  for (int mesh = 0; mesh < 2; ++mesh)
    for (int i = 0; i < 3; ++i)
      for (int a = 0; a < 3; ++a) e[mesh][i][a] = dsub(X[mesh][i + 1][a], X[mesh][0][a]);
  int fold = 0;
  double vol6[2];
  for (int mesh = 0; mesh < 2; ++mesh) {
    double r1[3];
    cross3d(e[mesh][1], e[mesh][2], r1);
    vol6[mesh] = dot3d(e[mesh][0], r1);
    if (!(vol6[mesh] > 0 && isfinite(vol6[mesh]))) ++fold;
  }
  for (int i = 0; i < 4; ++i) {
    uint8_t fm = pr.fixmask[vid[i]];
    for (int mesh = 0; mesh < 2; ++mesh) {
      int bad = 0;
      for (int a = 0; a < 3; ++a)
        if ((fm >> a) & 1) {
          double rv = ((fm >> (3 + a)) & 1) ? (double)pr.n[mesh][a] - 0.5 : -0.5;
          if (!(X[mesh][i][a] == rv)) bad = 1;
        }
      fold += bad;
    }
  }
  b.o_fold[tt] = fold;

  // deformation (FP32 from FP64 edge vectors and their differences)
  float es[3][3], dd[3][3];
  for (int i = 0; i < 3; ++i)
    for (int a = 0; a < 3; ++a) {
      es[i][a] = (float)e[0][i][a];
      dd[i][a] = (float)dsub(e[1][i][a], e[0][i][a]);
    }
  double def = 0.0;
  if (pr.model == 0) {
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

  // the two directions
  for (int d = 0; d < 2; ++d) {
    ItemRec& R = b.rec[2 * (size_t)tt + d];
    const double(*own)[3] = X[d];
    const double(*par)[3] = X[1 - d];
    const int* n = pr.n[d];
    const int* np = pr.n[1 - d];
    int flags = (vol6[d] > 0 && isfinite(vol6[d])) ? 1 : 0;
    R.prob = pi;
    R.tet = t;
    R.dir = d;
    // map (FP64, oracle formula): G = [D1 D2 D3][r1;r2;r3]/det
    double eo[3][3], D[3][3], r[3][3];
    for (int i = 0; i < 3; ++i)
      for (int a = 0; a < 3; ++a) {
        eo[i][a] = e[d][i][a];
        D[i][a] = dsub(e[1 - d][i][a], e[d][i][a]);
      }
    cross3d(eo[1], eo[2], r[0]);
    cross3d(eo[2], eo[0], r[1]);
    cross3d(eo[0], eo[1], r[2]);
    double det = dot3d(eo[0], r[0]);
    double inv = 1.0 / det;
    double G64[3][3];
    for (int c = 0; c < 3; ++c)
      for (int j = 0; j < 3; ++j)
        G64[c][j] = dmul(dadd(dmul(D[0][c], r[0][j]), dadd(dmul(D[1][c], r[1][j]), dmul(D[2][c], r[2][j]))), inv);
    for (int c = 0; c < 3; ++c) {
      for (int j = 0; j < 3; ++j) R.G64[c][j] = G64[c][j];
      R.d0[c] = dsub(par[0][c], own[0][c]);
    }
    for (int i = 0; i < 4; ++i)
      for (int a = 0; a < 3; ++a) R.X[i][a] = own[i][a];
    // linear-elastic energy from the source->target map (direction 0)
    if (d == 0 && pr.model == 1 && det != 0.0 && isfinite(det)) {
      float H[3][3];
      for (int c = 0; c < 3; ++c)
        for (int j = 0; j < 3; ++j) {
          float g = (float)G64[c][j] * pr.sp[1][c] / pr.sp[0][j];
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
    if (!flags) {
      R.flags = 0;
      for (int a = 0; a < 4; ++a) {
        R.b0[a] = 1;
        R.b1[a] = 0;
      }
      continue;
    }
    // bbox and origins
    double lo[3], hi[3], plo[3];
    for (int a = 0; a < 3; ++a) {
      lo[a] = hi[a] = own[0][a];
      plo[a] = par[0][a];
      for (int i = 1; i < 4; ++i) {
        lo[a] = fmin(lo[a], own[i][a]);
        hi[a] = fmax(hi[a], own[i][a]);
        plo[a] = fmin(plo[a], par[i][a]);
      }
    }
    int O[3], Op[3];
    int L = 1;
    for (int a = 0; a < 3; ++a) {
      double cl = ceil(lo[a]), fh = floor(hi[a]);
      int b0 = cl < 0 ? 0 : (int)fmin(cl, (double)n[a]);
      int b1 = fh > n[a] - 1 ? n[a] - 1 : (int)fmax(fh, -1.0);
      R.b0[a] = b0;
      R.b1[a] = b1;
      O[a] = (int)fmax(fmin(floor(lo[a]), (double)n[a]), -2.0);
      Op[a] = (int)fmax(fmin(floor(plo[a]), (double)np[a]), -2.0);
      R.O[a] = O[a];
      R.Op[a] = Op[a];
      L = max(L, b1 - O[a] + 1);
    }
    R.b0[3] = R.b1[3] = R.O[3] = R.Op[3] = 0;
    if (R.b0[0] > R.b1[0] || R.b0[1] > R.b1[1] || R.b0[2] > R.b1[2]) flags = 0;
    R.flags = flags;
    for (int i = 0; i < 4; ++i) {
      for (int a = 0; a < 3; ++a) R.vr[i][a] = (float)dsub(own[i][a], (double)O[a]);
      R.vr[i][3] = 0.f;
    }
    // faces: inward normal in FP32, offset, certified margin
    uint32_t fp = pr.fperm[t];
    for (int f = 0; f < 4; ++f) {
      int ia = face_local(fp, f, 0), ib = face_local(fp, f, 1), ic = face_local(fp, f, 2);
      int s = face_sign(fp, f);
      double u[3], w[3], nn[3], ar[3];
      for (int a = 0; a < 3; ++a) {
        u[a] = dsub(own[ib][a], own[ia][a]);
        w[a] = dsub(own[ic][a], own[ia][a]);
        ar[a] = dsub(own[ia][a], (double)O[a]);
      }
      cross3d(u, w, nn);
      double bp = -(double)s * dot3d(nn, ar);
      float Ax = (float)(s * nn[0]), Ay = (float)(s * nn[1]), Az = (float)(s * nn[2]);
      float Bp = (float)bp;
      float an = fabsf(Ax) + fabsf(Ay) + fabsf(Az);
      float uw = fabs3max((float)u[0], (float)u[1], (float)u[2]) * fabs3max((float)w[0], (float)w[1], (float)w[2]);
      float Lf = (float)(L + 1);
      float mu = 1.0f / 524288.0f * (an * Lf + fabsf(Bp)) + 1.5e-14f * (uw + an) * Lf + 1e-30f;
      R.fa[f][0] = Ax;
      R.fa[f][1] = Ay;
      R.fa[f][2] = Az;
      R.fa[f][3] = Bp;
      R.fm[f][0] = mu;
      R.fm[f][1] = 1.0f / Ax;
      R.fm[f][2] = 0.f;
      R.fm[f][3] = 0.f;
    }
    // FP32 map relative to the origins: p'_rel = vr + G vr + k
    double kk[3];
    double oo[3];
    for (int a = 0; a < 3; ++a) oo[a] = dsub((double)O[a], own[0][a]);
    float gmax = 0.f, kmax = 0.f;
    for (int c = 0; c < 3; ++c) {
      kk[c] = dadd(dadd((double)(O[c] - Op[c]), R.d0[c]),
                   dadd(dmul(G64[c][0], oo[0]), dadd(dmul(G64[c][1], oo[1]), dmul(G64[c][2], oo[2]))));
      for (int j = 0; j < 3; ++j) {
        R.G[c][j] = (float)G64[c][j];
        gmax = fmaxf(gmax, fabsf(R.G[c][j]));
      }
      R.G[c][3] = (float)kk[c];
      kmax = fmaxf(kmax, fabsf(R.G[c][3]));
    }
    float M = (float)L * (1.0f + 3.0f * gmax) + kmax + 2.0f;
    R.gx[0] = 1.0f + R.G[0][0];
    R.gx[1] = R.G[1][0];
    R.gx[2] = R.G[2][0];
    R.gx[3] = M * (1.0f / 524288.0f);  // black-decision margin delta (2^-19 M)
    for (int a = 0; a < 3; ++a) {
      R.clo[a] = (float)(-1 - Op[a]);
      R.chi[a] = (float)(np[a] - Op[a]);
    }
    R.clo[3] = R.chi[3] = 0.f;
    // corner-cell index: cell (i,j,k) with i = Op.x + floor(p'_rel.x) etc.
    unsigned Sy = (unsigned)(np[0] + 2), Sz = (unsigned)((np[1] + 2) * (np[0] + 2));
    unsigned base = ((unsigned)(Op[2] + 1) * (unsigned)(np[1] + 2) + (unsigned)(Op[1] + 1)) * Sy + (unsigned)(Op[0] + 1);
    base -= (unsigned)MAGIC_BITS * (Sz + Sy + 1u);
    R.cbase = base;
  }
  b.o_def[tt] = def;
}

void launch_setup(const DevProblem* probs, const Batch& b, cudaStream_t st) {
  if (b.n_tt <= 0) return;
  k_setup<<<(b.n_tt + 127) / 128, 128, 0, st>>>(probs, b);
}

// ------------------------------------------------------------ raster + sample
struct WarpSmem {
  ItemRec rec;
  int2 meta[32];     // (excl prefix, own plain index of x0)
  float4 pr0[32];    // mapped partner-relative coordinate of x0
};

__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(FULL_MASK, v, o);
    if (lane >= o) v += y;
  }
  return v;
}

// y-range of slice z (relative to O) through the tet: min/max over edges
// crossing the plane; a superset (slack) of the rows holding inside voxels.
__device__ __forceinline__ void slice_yrange(const ItemRec& r, float zr, float& ylo, float& yhi) {
  ylo = 3.0e38f;
  yhi = -3.0e38f;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = i + 1; j < 4; ++j) {
      float zi = r.vr[i][2], zj = r.vr[j][2];
      float yi = r.vr[i][1], yj = r.vr[j][1];
      if ((zi - zr) * (zj - zr) <= 0.f) {
        float y;
        if (zj != zi) {
          float tq = (zr - zi) / (zj - zi);
          tq = fminf(fmaxf(tq, 0.f), 1.f);
          y = fmaf(tq, yj - yi, yi);
          ylo = fminf(ylo, y);
          yhi = fmaxf(yhi, y);
        } else {
          ylo = fminf(ylo, fminf(yi, yj));
          yhi = fmaxf(yhi, fmaxf(yi, yj));
        }
      }
    }
}

// Exact span of row (y, z): x range (relative to O) inside all 4 faces.
// Returns false when the row is empty.  Rows where the FP32 margin cannot
// decide a face take the careful path: every voxel of the row range is
// classified face by face, exactly where the margin does not decide.
__device__ __noinline__ void span_careful(const ItemRec& r, uint32_t fp, int xl, int xh, int yi, int zi,
                                          int& lo, int& hi) {
  const float yr = (float)yi, zr = (float)zi;
  int first = xh + 1, last = xl - 1;
  for (int x = xl; x <= xh; ++x) {
    bool in = true;
    for (int f = 0; f < 4 && in; ++f) {
      float c = fmaf(r.fa[f][1], yr, fmaf(r.fa[f][2], zr, r.fa[f][3]));
      float h = fmaf(r.fa[f][0], (float)x, c);
      float mu = r.fm[f][0];
      if (h > mu) continue;
      if (h < -mu) {
        in = false;
        break;
      }
      double p[3] = {(double)(x + r.O[0]), (double)(yi + r.O[1]), (double)(zi + r.O[2])};
      in = rec_face_in_exact(r, fp, f, p);
    }
    if (in) {
      first = min(first, x);
      last = max(last, x);
    }
  }
  lo = first;
  hi = last;
}

__device__ __forceinline__ void row_span(const ItemRec& r, uint32_t fp, int xl, int xh, int yi, int zi, int& lo,
                                         int& hi) {
  const float yr = (float)yi, zr = (float)zi;
  lo = xl;
  hi = xh;
  bool ok = true;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    float Ax = r.fa[f][0];
    float c = fmaf(r.fa[f][1], yr, fmaf(r.fa[f][2], zr, r.fa[f][3]));
    float mu = r.fm[f][0];
    if (Ax == 0.f) {
      if (c < -mu) hi = xl - 1;
      else if (!(c > mu)) ok = false;
      continue;
    }
    float th = -c * r.fm[f][1];
    th = fminf(fmaxf(th, (float)(xl - 1)), (float)(xh + 1));
    int kb;
    float kf = ffloor_magic(th, kb);
    int kint = kb - MAGIC_BITS;
    float h0 = fmaf(Ax, kf, c);
    float h1 = fmaf(Ax, kf + 1.0f, c);
    if (Ax > 0.f) {
      ok = ok && (kint < xl || h0 < -mu) && (kint + 1 > xh || h1 > mu);
      lo = max(lo, kint + 1);
    } else {
      ok = ok && (kint < xl || h0 > mu) && (kint + 1 > xh || h1 < -mu);
      hi = min(hi, kint);
    }
  }
  if (!ok) span_careful(r, fp, xl, xh, yi, zi, lo, hi);
}

// Black decision of one sample where the FP32 cell cannot decide it: FP64
// mapped coordinate (definition), its support, and the plain partner image.
__device__ __noinline__ bool black_exact(const ItemRec& r, const DevProblem& pr, int x, int y, int z) {
  double v[3] = {(double)x, (double)y, (double)z};
  double p[3];
  map_exact(r, v, p);
  int dp = 1 - r.dir;
  const int* n = pr.n[dp];
  int i0[3], i1[3];
  bool sup1[3];
  for (int a = 0; a < 3; ++a) {
    double q = fmin(fmax(p[a], -1.0), (double)n[a]);
    double fl = floor(q);
    int i = (int)fl;
    sup1[a] = (q - fl) > 0;
    i0[a] = min(max(i, 0), n[a] - 1);
    i1[a] = min(max(i + 1, 0), n[a] - 1);
  }
  for (int c = 0; c < 8; ++c) {
    int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
    if ((dx && !sup1[0]) || (dy && !sup1[1]) || (dz && !sup1[2])) continue;
    long li = ((long)(dz ? i1[2] : i0[2]) * n[1] + (dy ? i1[1] : i0[1])) * n[0] + (dx ? i1[0] : i0[0]);
    if (load_plain_dyn(pr.plain[dp], pr.dtype, li) != 0.0f) return false;
  }
  return true;
}

template <int ST, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_raster(const DevProblem* __restrict__ probs, Batch b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WarpSmem* ws = (WarpSmem*)smem_raw + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const unsigned lemask = 0xffffffffu >> (31 - lane);
  const int n_items = 2 * b.n_tt;
  for (;;) {
    int item = 0;
    if (lane == 0) item = (int)atomicAdd(b.work, 1u);
    item = __shfl_sync(FULL_MASK, item, 0);
    if (item >= n_items) break;
    // stage the record in shared memory
    {
      const int4* src = (const int4*)(b.rec + item);
      int4* dst = (int4*)&ws->rec;
      constexpr int NW = sizeof(ItemRec) / 16;
      for (int i = lane; i < NW; i += 32) dst[i] = __ldg(src + i);
    }
    __syncwarp();
    const ItemRec& r = ws->rec;
    float sum = 0.f, comp = 0.f;
    int cov = 0;
    if (r.flags & 1) {
      const DevProblem& pr = probs[r.prob];
      const int d = r.dir;
      const uint32_t fp = pr.fperm[r.tet];
      const void* own_img = pr.plain[d];
      const void* cells = pr.cells[1 - d];
      const uint8_t* cflag = pr.cflag[1 - d];
      const int nxo = pr.n[d][0], nyo = pr.n[d][1];
      const int Sy = pr.n[1 - d][0] + 2, Sz = (pr.n[1 - d][1] + 2) * Sy;
      const bool black = pr.black_rule != 0;
      const float G00 = r.G[0][0], G01 = r.G[0][1], G02 = r.G[0][2], K0 = r.G[0][3];
      const float G10 = r.G[1][0], G11 = r.G[1][1], G12 = r.G[1][2], K1 = r.G[1][3];
      const float G20 = r.G[2][0], G21 = r.G[2][1], G22 = r.G[2][2], K2 = r.G[2][3];
      const float gxx = r.gx[0], gxy = r.gx[1], gxz = r.gx[2], delta = r.gx[3];
      const float clx = r.clo[0], cly = r.clo[1], clz = r.clo[2];
      const float chx = r.chi[0], chy = r.chi[1], chz = r.chi[2];
      const unsigned cbase = r.cbase;
      const int Ox = r.O[0], Oy = r.O[1], Oz = r.O[2];
      const int xl = r.b0[0] - Ox, xh = r.b1[0] - Ox;
      const int by0 = r.b0[1], by1 = r.b1[1];
      for (int zb = r.b0[2]; zb <= r.b1[2]; zb += 32) {
        // slices -> y ranges
        int z = zb + lane;
        int ycnt = 0, ylo = 0;
        if (z <= r.b1[2]) {
          float ylf, yhf;
          slice_yrange(r, (float)(z - Oz), ylf, yhf);
          float slack = 1.0f / 256.0f + 1e-5f * fabsf(yhf);
          int y0 = max(by0, (int)ceilf(ylf - slack) + Oy);
          int y1 = min(by1, (int)floorf(yhf + slack) + Oy);
          if (ylf <= yhf && y1 >= y0) {
            ylo = y0;
            ycnt = y1 - y0 + 1;
          }
        }
        int yincl = warp_incl_scan(ycnt, lane);
        int yexcl = yincl - ycnt;
        const int R = __shfl_sync(FULL_MASK, yincl, 31);
        for (int rb = 0; rb < R; rb += 32) {
          const int rr = rb + lane;
          const bool has_row = rr < R;
          const int rq = has_row ? rr : R - 1;
          // slice holding row rq: the last lane with yexcl <= rq
          int s = 0;
#pragma unroll
          for (int step = 16; step > 0; step >>= 1) {
            const int cs = s + step;
            const int e = __shfl_sync(FULL_MASK, yexcl, cs & 31);
            if (cs < 32 && e <= rq) s = cs;
          }
          const int e_s = __shfl_sync(FULL_MASK, yexcl, s);
          const int yl_s = __shfl_sync(FULL_MASK, ylo, s);
          const int zrow = zb + s;
          const int yrow = yl_s + (rq - e_s);
          int xcnt = 0, x0 = 0;
          if (has_row) {
            int lo, hi;
            row_span(r, fp, xl, xh, yrow - Oy, zrow - Oz, lo, hi);
            if (hi >= lo) {
              xcnt = hi - lo + 1;
              x0 = lo + Ox;
            }
          }
          // compact non-empty rows and publish them
          const unsigned nz = __ballot_sync(FULL_MASK, xcnt > 0);
          const int cidx = __popc(nz & (lemask >> 1));
          const int xincl = warp_incl_scan(xcnt, lane);
          const int xexcl = xincl - xcnt;
          const int T = __shfl_sync(FULL_MASK, xincl, 31);
          if (xcnt > 0) {
            float vx = (float)(x0 - Ox), vy = (float)(yrow - Oy), vz = (float)(zrow - Oz);
            float px = vx + fmaf(G00, vx, fmaf(G01, vy, fmaf(G02, vz, K0)));
            float py = vy + fmaf(G10, vx, fmaf(G11, vy, fmaf(G12, vz, K1)));
            float pz = vz + fmaf(G20, vx, fmaf(G21, vy, fmaf(G22, vz, K2)));
            ws->meta[cidx] = make_int2(xexcl, (zrow * nyo + yrow) * nxo + x0);
            ws->pr0[cidx] = make_float4(px, py, pz, 0.f);
          }
          __syncwarp();
          int rows_before = 0;
          for (int vb = 0; vb < T; vb += 32) {
            unsigned bit = (xcnt > 0 && xexcl >= vb && xexcl < vb + 32) ? (1u << (xexcl - vb)) : 0u;
            const unsigned sm = __reduce_or_sync(FULL_MASK, bit);
            const int v = vb + lane;
            const int row = rows_before + __popc(sm & lemask) - 1;
            rows_before += __popc(sm);
            if (v < T) {
              const int2 mt = ws->meta[row];
              const float4 p0 = ws->pr0[row];
              const int dx = v - mt.x;
              const float dxf = __int_as_float(dx + MAGIC_BITS) - MAGIC;
              float px = fminf(fmaxf(fmaf(dxf, gxx, p0.x), clx), chx);
              float py = fminf(fmaxf(fmaf(dxf, gxy, p0.y), cly), chy);
              float pz = fminf(fmaxf(fmaf(dxf, gxz, p0.z), clz), chz);
              int ix, iy, iz;
              float flx = ffloor_magic(px, ix), fly = ffloor_magic(py, iy), flz = ffloor_magic(pz, iz);
              float fx = px - flx, fy = py - fly, fz = pz - flz;
              unsigned cidx2 = cbase + (unsigned)iz * (unsigned)Sz + (unsigned)iy * (unsigned)Sy + (unsigned)ix;
              float s = cell_lerp<ST>(cells, cidx2, fx, fy, fz);
              float o = load_plain<ST>(own_img, mt.y + dx);
              float dd = o - s;
              float d2 = dd * dd;
              if (black) {
                const uint8_t cf = __ldg(cflag + cidx2);
                bool own0 = (o == 0.0f);
                bool blk = false;
                if (cf & 1) {
                  bool nearp = fminf(fminf(fx, fy), fz) < delta || fmaxf(fmaxf(fx, fy), fz) > 1.0f - delta;
                  if (!nearp) {
                    blk = (cf & 2) != 0;
                  } else {
                    const int xa = (mt.y + dx) % nxo;
                    const int rem = (mt.y + dx) / nxo;
                    blk = black_exact(r, pr, xa, rem % nyo, rem / nyo);
                  }
                }
                if (own0 != blk) d2 = 1.0f;
              }
              // Kahan
              float yk = d2 - comp;
              float tk = sum + yk;
              comp = (tk - sum) - yk;
              sum = tk;
              ++cov;
            }
          }
          __syncwarp();
        }
      }
    }
    // error-free warp reduction of (sum, -comp)
    float hi = sum, lo = -comp;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float oh = __shfl_xor_sync(FULL_MASK, hi, o);
      float ol = __shfl_xor_sync(FULL_MASK, lo, o);
      float sh = hi + oh;
      float bb = sh - hi;
      float err = (hi - (sh - bb)) + (oh - bb);
      hi = sh;
      lo = lo + ol + err;
    }
    int covt = __reduce_add_sync(FULL_MASK, cov);
    if (lane == 0) {
      b.o_ssd[item] = (double)hi + (double)lo;
      b.o_cov[item] = covt;
    }
    __syncwarp();
  }
}

void launch_raster(const DevProblem* probs, const Batch& b, int st_dtype, int warps, int vpw, int n_sm,
                   cudaStream_t st) {
  (void)vpw;
  if (b.n_tt <= 0) return;
  int threads = 32 * warps;
  size_t smem = sizeof(WarpSmem) * warps;
  long items = 2L * b.n_tt;
  int per_sm = 2048 / threads;
  long blocks = (long)n_sm * per_sm;
  long need = (items + warps - 1) / warps;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
#define DMR_RASTER_LAUNCH(ST_, W_) k_raster<ST_, W_><<<(unsigned)blocks, threads, smem, st>>>(probs, b)
#define DMR_RASTER_BY_WARPS(ST_)          \
  if (warps == 4) DMR_RASTER_LAUNCH(ST_, 4);  \
  else if (warps == 16) DMR_RASTER_LAUNCH(ST_, 16); \
  else DMR_RASTER_LAUNCH(ST_, 8)
  if (st_dtype == ST_F32) {
    DMR_RASTER_BY_WARPS(ST_F32);
  } else if (st_dtype == ST_BF16) {
    DMR_RASTER_BY_WARPS(ST_BF16);
  } else {
    DMR_RASTER_BY_WARPS(ST_F16);
  }
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
    float mu = r.fm[f][0] + an * (pmag + fabsf(px) + fabsf(py) + fabsf(pz) + 1.0f) * (1.0f / 1048576.0f);
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

__device__ double landmark_term(const ItemRec& r, const DevProblem& pr, const double p[3], const double q[3]) {
  double pm[3];
  map_exact(r, p, pm);
  int dp = 1 - r.dir;
  double s = 0.0;
  for (int a = 0; a < 3; ++a) {
    double d = dmul(dsub(pm[a], q[a]), pr.spd[dp][a]);
    s = dadd(s, dmul(d, d));
  }
  return s;
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
  double p[3], q[3];
  for (int a = 0; a < 3; ++a) {
    p[a] = pr.guide[6 * i + 3 * mesh + a];
    q[a] = pr.guide[6 * i + 3 * (1 - mesh) + a];
  }
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
    pr.c_gterm[li] = found >= 0 ? landmark_term(b.rec[2 * ((size_t)ci * pr.ntet + found) + mesh], pr, p, q) : 0.0;
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
__global__ void k_landmarks_partial(const DevProblem* probs, Batch b) {
  int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (k >= b.n_trials) return;
  const DevProblem& pr = probs[b.tr_prob ? b.tr_prob[k] : 0];
  const int ng = pr.ng;
  const int cand = b.tr_cand[k];
  const int first = b.tr_first[k], ntt = b.tr_ntt[k];
  const int* tl = b.tt_tet + first;
  int naff = 0;
  double gd = 0.0;
  int ud = 0;
  for (int base = 0; base < 2 * ng; base += 32) {
    int e = base + lane;
    bool aff = false;
    int told = -2;
    if (e < 2 * ng) {
      int mesh = e / ng, i = e % ng;
      told = pr.c_loc[((size_t)cand * 2 + mesh) * ng + i];
      if (told < 0) aff = true;
      else {
        int lo = 0, hi = ntt - 1;
        while (lo <= hi) {
          int mid = (lo + hi) >> 1;
          int v = tl[mid];
          if (v == told) {
            aff = true;
            break;
          }
          if (v < told) lo = mid + 1;
          else hi = mid - 1;
        }
      }
    }
    unsigned am = __ballot_sync(FULL_MASK, aff);
    while (am) {
      int src = __ffs(am) - 1;
      am &= am - 1;
      int ee = base + src;
      int mesh = ee / ng, i = ee % ng;
      int t_old = __shfl_sync(FULL_MASK, told, src);
      double p[3], q[3];
      for (int a = 0; a < 3; ++a) {
        p[a] = pr.guide[6 * i + 3 * mesh + a];
        q[a] = pr.guide[6 * i + 3 * (1 - mesh) + a];
      }
      float pmag = fmaxf(fabsf((float)p[0]), fmaxf(fabsf((float)p[1]), fabsf((float)p[2])));
      int found = -1;
      for (int jb = 0; jb < ntt && found < 0; jb += 32) {
        int j = jb + lane;
        bool in = false;
        if (j < ntt) {
          const ItemRec& r = b.rec[2 * (size_t)(first + j) + mesh];
          in = lm_test(r, pr.fperm[tl[j]], p, pmag);
        }
        unsigned m = __ballot_sync(FULL_MASK, in);
        if (m) found = jb + __ffs(m) - 1;
      }
      if (lane == 0) {
        double term = found >= 0 ? landmark_term(b.rec[2 * (size_t)(first + found) + mesh], pr, p, q) : 0.0;
        size_t li = ((size_t)cand * 2 + mesh) * ng + i;
        double old = pr.c_gterm[li];
        gd = dadd(gd, dsub(term, old));
        ud += (found < 0 ? 1 : 0) - (t_old < 0 ? 1 : 0);
        if (naff < b.aff_cap) {
          size_t o = (size_t)k * b.aff_cap + naff;
          b.aff_idx[o] = ee;
          b.aff_loc[o] = found >= 0 ? tl[found] : -1;
          b.aff_term[o] = term;
        }
        ++naff;
      }
    }
  }
  if (lane == 0) {
    b.aff_n[k] = min(naff, b.aff_cap);
    b.tr_delta[4 * (size_t)k + 2] = gd;
    b.tr_delta[4 * (size_t)k + 3] = (double)ud;
  }
}

void launch_landmarks_partial(const DevProblem* probs, const Batch& b, cudaStream_t st) {
  if (b.n_trials <= 0) return;
  long threads = 32L * b.n_trials;
  k_landmarks_partial<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(probs, b);
}

// Partial evaluation: new = stored - sum old + sum new over touched tets.
__global__ void k_reduce_partial(const DevProblem* probs, Batch b, int has_landmarks) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= b.n_trials) return;
  const DevProblem& pr = probs[b.tr_prob ? b.tr_prob[k] : 0];
  const int cand = b.tr_cand[k];
  const int first = b.tr_first[k], ntt = b.tr_ntt[k];
  double old[3] = {0, 0, 0}, nw[3] = {0, 0, 0};
  unsigned long long cov = 0;
  for (int j = 0; j < ntt; ++j) {
    int tt = first + j;
    size_t ci = (size_t)cand * pr.ntet + b.tt_tet[tt];
    old[0] = dadd(old[0], dadd(pr.c_ssd[2 * ci], pr.c_ssd[2 * ci + 1]));
    old[1] = dadd(old[1], pr.c_def[ci]);
    old[2] = dadd(old[2], (double)pr.c_fold[ci]);
    nw[0] = dadd(nw[0], dadd(b.o_ssd[2 * (size_t)tt], b.o_ssd[2 * (size_t)tt + 1]));
    nw[1] = dadd(nw[1], b.o_def[tt]);
    nw[2] = dadd(nw[2], (double)b.o_fold[tt]);
    cov += (unsigned)(b.o_cov[2 * (size_t)tt] + b.o_cov[2 * (size_t)tt + 1]);
  }
  double* dl = b.tr_delta + 4 * (size_t)k;
  dl[0] = dsub(nw[0], old[0]);
  dl[1] = dsub(nw[1], old[1]);
  double gd = has_landmarks ? dl[2] : 0.0;
  double ud = has_landmarks ? dl[3] : 0.0;
  if (!has_landmarks) dl[2] = 0.0;
  dl[3] = dadd(dsub(nw[2], old[2]), ud);
  const double* s = pr.sums + 4 * (size_t)cand;
  double* ob = b.tr_obj + 4 * (size_t)k;
  ob[0] = dadd(s[0], dl[0]) / pr.sim_norm;
  ob[1] = dadd(s[1], dl[1]) / pr.def_norm;
  ob[2] = pr.ng > 0 ? dadd(s[2], gd) / pr.guid_norm : 0.0;
  ob[3] = dadd(s[3], dl[3]);
  atomicAdd(pr.samples, cov);
}

void launch_reduce_partial(const DevProblem* probs, const Batch& b, cudaStream_t st) {
  if (b.n_trials <= 0) return;
  k_reduce_partial<<<(b.n_trials + 127) / 128, 128, 0, st>>>(probs, b, b.aff_n != nullptr);
}

// Accept-if-improves (Sec. 2.2), constraint domination first.
__global__ void k_accept(const DevProblem* probs, Batch b, uint8_t* accept) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= b.n_trials) return;
  const DevProblem& pr = probs[b.tr_prob ? b.tr_prob[k] : 0];
  const double* s = pr.sums + 4 * (size_t)b.tr_cand[k];
  const double* o = b.tr_obj + 4 * (size_t)k;
  double cur[4] = {s[0] / pr.sim_norm, s[1] / pr.def_norm, pr.ng > 0 ? s[2] / pr.guid_norm : 0.0, s[3]};
  bool acc;
  if (o[3] != cur[3]) acc = o[3] < cur[3];
  else {
    bool le = o[0] <= cur[0] && o[1] <= cur[1] && o[2] <= cur[2];
    bool lt = o[0] < cur[0] || o[1] < cur[1] || o[2] < cur[2];
    acc = le && lt;
  }
  accept[k] = acc ? 1 : 0;
}

void launch_accept(const DevProblem* probs, const Batch& b, uint8_t* accept, cudaStream_t st) {
  if (b.n_trials <= 0) return;
  k_accept<<<(b.n_trials + 127) / 128, 128, 0, st>>>(probs, b, accept);
}

// Commit: per touched tet (cache), per trial (coords, landmarks), per
// candidate (ordered sum of accepted deltas).
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

__global__ void k_commit_sums(const DevProblem* probs, Batch b, const uint8_t* accept, const int* cand_ptr,
                              const int* cand_trials, int n_list) {
  int ci = blockIdx.x * blockDim.x + threadIdx.x;
  if (ci >= n_list) return;
  int k0 = cand_trials[cand_ptr[ci]];
  const DevProblem& pr = probs[b.tr_prob ? b.tr_prob[k0] : 0];
  double* s = pr.sums + 4 * (size_t)b.tr_cand[k0];
  for (int j = cand_ptr[ci]; j < cand_ptr[ci + 1]; ++j) {
    int k = cand_trials[j];
    if (!accept[k]) continue;
    for (int q = 0; q < 4; ++q) s[q] = dadd(s[q], b.tr_delta[4 * (size_t)k + q]);
  }
}

void launch_commit(const DevProblem* probs, const Batch& b, const uint8_t* accept, const int* tr_group,
                   const int* g_ptr, const int* g_pts, const int* cand_ptr, const int* cand_trials, int n_list,
                   cudaStream_t st) {
  if (b.n_trials <= 0) return;
  k_commit_tt<<<(b.n_tt + 255) / 256, 256, 0, st>>>(probs, b, accept);
  k_commit_trial<<<b.n_trials, 64, 0, st>>>(probs, b, accept, tr_group, g_ptr, g_pts);
  k_commit_sums<<<(n_list + 127) / 128, 128, 0, st>>>(probs, b, accept, cand_ptr, cand_trials, n_list);
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
