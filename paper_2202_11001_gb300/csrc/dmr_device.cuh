// Device-side helpers shared by the kernels of the GB300 evaluator, and the
// rasterise-and-sample kernel template (instantiated per image storage type
// in dmr_raster_{f32,bf16,f16}.cu so the three compile in parallel).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "dmr_internal.cuh"

namespace dmr {

#define FULL_MASK 0xffffffffu

// ------------------------------------------------------------ FP64 exact
static __device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
static __device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
static __device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }

static __device__ __forceinline__ void cross3d(const double a[3], const double b[3], double o[3]) {
  o[0] = dsub(dmul(a[1], b[2]), dmul(a[2], b[1]));
  o[1] = dsub(dmul(a[2], b[0]), dmul(a[0], b[2]));
  o[2] = dsub(dmul(a[0], b[1]), dmul(a[1], b[0]));
}
static __device__ __forceinline__ double dot3d(const double a[3], const double b[3]) {
  return dadd(dmul(a[0], b[0]), dadd(dmul(a[1], b[1]), dmul(a[2], b[2])));
}

// Conversions that keep the FP64 pipe free: on GB300 double arithmetic and
// double <-> float / int conversions all issue at under 2 operations per SM
// clock (FP32 arithmetic: over 100), so a kernel bound by its FP64 work
// converts in integer arithmetic instead.  d2f: IEEE-754 binary64 -> binary32
// with round-to-nearest-even, written out for results in the normal binary32
// range (the 23 leading fraction bits, the 29 dropped bits decide the
// rounding, a carry runs into the exponent and past the largest finite value
// to infinity); zeros, subnormal results, infinities and NaN take the
// hardware conversion.
static __device__ __forceinline__ float d2f(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned ex = (hi >> 20) & 0x7ffu;
  if (ex - 897u > 253u) return __double2float_rn(x);
  unsigned f = ((ex - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned r = lo & 0x1fffffffu;
  f += (r > 0x10000000u || (r == 0x10000000u && (f & 1u))) ? 1u : 0u;
  return __uint_as_float((hi & 0x80000000u) | f);
}
// i2d: the exact binary64 value of a 32-bit integer (leading one found by
// counting leading zeros, the bits below it become the fraction).
static __device__ __forceinline__ double i2d(int v) {
  if (v == 0) return 0.0;
  const unsigned s = v < 0 ? 0x80000000u : 0u;
  const unsigned a = v < 0 ? 0u - (unsigned)v : (unsigned)v;
  const int lz = __clz(a);
  const unsigned fr = a << lz << 1;  // two shifts: lz + 1 may be 32
  return __hiloint2double((int)(s | ((unsigned)(1054 - lz) << 20) | (fr >> 12)), (int)(fr << 20));
}

// Exact face predicate: canonical face (a,b,c) with inward sign s; p on the
// inner side, or on the plane and the signed normal's first nonzero
// component in (z, y, x) order is positive.
static __device__ __noinline__ bool face_in_exact(const double* A, const double* B, const double* Cc, int s,
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

static __device__ __forceinline__ int face_local(uint32_t fp, int f, int which) { return (fp >> (8 * f + 2 * which)) & 3; }
static __device__ __forceinline__ int face_sign(uint32_t fp, int f) { return ((fp >> (8 * f + 6)) & 1) ? -1 : 1; }

// Exact face test of face f of the record's own tet at point p.
static __device__ __forceinline__ bool rec_face_in_exact(const ItemRec& r, uint32_t fp, int f, const double p[3]) {
  int ia = face_local(fp, f, 0), ib = face_local(fp, f, 1), ic = face_local(fp, f, 2);
  return face_in_exact(r.X[ia], r.X[ib], r.X[ic], face_sign(fp, f), p);
}

// FP64 mapped coordinate, the definition the black decision follows:
// p' = (v + d0) + G (v - own_0) with G = [D1 D2 D3][r1; r2; r3] / det
// (Sec. 2.3.1), every operation in the oracle's order, rebuilt from the own
// and partner vertices of the record (only decisions the FP32 path cannot
// certify come here).
static __device__ __noinline__ void map_exact(const ItemRec& r, const double v[3], double out[3]) {
  double e[3][3], D[3][3], rr[3][3];
  for (int i = 0; i < 3; ++i)
    for (int a = 0; a < 3; ++a) {
      e[i][a] = dsub(r.X[i + 1][a], r.X[0][a]);
      D[i][a] = dsub(dsub(r.XP[i + 1][a], r.XP[0][a]), e[i][a]);
    }
  cross3d(e[1], e[2], rr[0]);
  cross3d(e[2], e[0], rr[1]);
  cross3d(e[0], e[1], rr[2]);
  const double inv = 1.0 / dot3d(e[0], rr[0]);
  double q[3];
  for (int a = 0; a < 3; ++a) q[a] = dsub(v[a], r.X[0][a]);
  for (int c = 0; c < 3; ++c) {
    double G[3];
    for (int j = 0; j < 3; ++j)
      G[j] = dmul(dadd(dmul(D[0][c], rr[0][j]), dadd(dmul(D[1][c], rr[1][j]), dmul(D[2][c], rr[2][j]))), inv);
    out[c] = dadd(dadd(v[c], dsub(r.XP[0][c], r.X[0][c])),
                  dadd(dmul(G[0], q[0]), dadd(dmul(G[1], q[1]), dmul(G[2], q[2]))));
  }
}

// ------------------------------------------------------------ float helpers
#define MAGIC 12582912.0f /* 1.5 * 2^23 */
#define MAGIC_BITS 0x4B400000

// floor for |x| < 2^22 with two full-rate ALU ops: returns the float floor
// and the integer floor + MAGIC_BITS (as raw bits).
static __device__ __forceinline__ float ffloor_magic(float x, int& ibits) {
  float t = __fadd_rd(x, MAGIC);
  ibits = __float_as_int(t);
  return t - MAGIC;
}

static __device__ __forceinline__ float bf16lo(uint32_t w) { return __uint_as_float(w << 16); }
static __device__ __forceinline__ float bf16hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
static __device__ __forceinline__ float f16lo(uint32_t w) { return __half2float(__ushort_as_half((unsigned short)(w & 0xffff))); }
static __device__ __forceinline__ float f16hi(uint32_t w) { return __half2float(__ushort_as_half((unsigned short)(w >> 16))); }

template <int ST>
static __device__ __forceinline__ float load_plain(const void* p, long i) {
  if (ST == ST_F32) return __ldg((const float*)p + i);
  unsigned short u = __ldg((const unsigned short*)p + i);
  if (ST == ST_BF16) return __uint_as_float((uint32_t)u << 16);
  return __half2float(__ushort_as_half(u));
}

static __device__ __forceinline__ float load_plain_dyn(const void* p, int st, long i) {
  if (st == ST_F32) return load_plain<ST_F32>(p, i);
  if (st == ST_BF16) return load_plain<ST_BF16>(p, i);
  return load_plain<ST_F16>(p, i);
}

static __device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(FULL_MASK, v, o);
    if (lane >= o) v += y;
  }
  return v;
}

// Shared-memory load of 4 floats that the compiler may not hoist or merge:
// the record stays in shared memory instead of occupying registers across
// the row and voxel loops.
static __device__ __forceinline__ float4 lds4(const float* p) {
  float4 v;
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
  return v;
}

// y-range of slice z (relative to O) through the tet: min/max over edges
// crossing the plane; a superset (slack) of the rows holding inside voxels.
static __device__ __forceinline__ void slice_yrange(const ItemRec& r, float zr, float& ylo, float& yhi) {
  ylo = 3.0e38f;
  yhi = -3.0e38f;
  float4 v[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = lds4(&r.vr[i][0]);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = i + 1; j < 4; ++j) {
      float zi = v[i].z, zj = v[j].z;
      float yi = v[i].y, yj = v[j].y;
      if ((zi - zr) * (zj - zr) <= 0.f) {
        float y;
        if (zj != zi) {
          // the range only needs to contain the rows (the caller widens it
          // by a slack of 1/256 + 1e-5 |y|), so an approximate quotient
          // (a few ulp) serves
          float tq = __fdividef(zr - zi, zj - zi);
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

// Exact span of row (y, z): x range (relative to O) inside all 4 faces, for
// rows where the FP32 margins cannot certify the fast span.  For a fixed row
// the FP64 face predicate is monotone in x (every rounding step is), with
// direction sign(s n_x), and the tie rule is constant per face; so each
// face's inside set is a prefix or suffix of the row, and the row's span is
// an interval.  Where |A.x| exceeds the bound on its rounding error (fm[3])
// the direction is sign(A.x): walk from the FP32 threshold to the exact
// boundary, deciding each voxel with the margin and, inside it, with the
// FP64 predicate.  Otherwise scan the row for that face.
static __device__ __noinline__ void span_careful(const ItemRec& r, uint32_t fp, int xl, int xh, int yi, int zi,
                                                 int& lo, int& hi) {
  const float yr = (float)yi, zr = (float)zi;
  const double py = (double)(yi + r.O[1]), pz = (double)(zi + r.O[2]);
  lo = xl;
  hi = xh;
  for (int f = 0; f < 4 && lo <= hi; ++f) {
    const float Ax = r.fa[f][0];
    const float c = fmaf(r.fa[f][1], yr, fmaf(r.fa[f][2], zr, r.fa[f][3]));
    const float mu = r.fm[f][0];
    auto in_f = [&](int x) -> bool {
      const float h = fmaf(Ax, (float)x, c);
      if (h > mu) return true;
      if (h < -mu) return false;
      const double p[3] = {(double)(x + r.O[0]), py, pz};
      return rec_face_in_exact(r, fp, f, p);
    };
    if (fabsf(Ax) > r.fm[f][3]) {
      const float th = fminf(fmaxf(-c * r.fm[f][1], (float)(lo - 1)), (float)(hi + 1));
      const int k = (int)floorf(th);
      if (Ax > 0.f) {
        int xs = min(max(k + 1, lo), hi + 1);
        while (xs > lo && in_f(xs - 1)) --xs;
        while (xs <= hi && !in_f(xs)) ++xs;
        lo = xs;
      } else {
        int xe = min(max(k, lo - 1), hi);
        while (xe < hi && in_f(xe + 1)) ++xe;
        while (xe >= lo && !in_f(xe)) --xe;
        hi = xe;
      }
    } else {
      int first = hi + 1, last = lo - 1;
      for (int x = lo; x <= hi; ++x)
        if (in_f(x)) {
          first = min(first, x);
          last = x;
        }
      lo = first;
      hi = last;
    }
  }
}

// Exact span of row (y, z), x relative to O.  Every face's FP32 threshold
// gives a candidate span; the span is accepted only if the margins certify
// it: all voxels of [lo, hi] certainly inside every face, and the voxel just
// outside each end certainly outside its binding face (h is monotone in x,
// so that settles the whole row).  Otherwise the careful path decides.
template <bool FAST>
static __device__ __forceinline__ void row_span(const ItemRec& r, uint32_t fp, int xl, int xh, int yi, int zi,
                                                int& lo, int& hi, bool& careful) {
  const float yr = (float)yi, zr = (float)zi;
  lo = xl;
  hi = xh;
  bool ok = true;
  // binding faces of the two ends: (A.x, h at x = 0, margin)
  float Al = 0.f, cl = 0.f, ml = 0.f, Ah = 0.f, ch = 0.f, mh = 0.f;
  bool hasl = false, hash = false;
  float Av[4], cv[4], mv[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const float4 A = lds4(&r.fa[f][0]);
    const float4 M = lds4(&r.fm[f][0]);
    Av[f] = A.x;
    cv[f] = fmaf(A.y, yr, fmaf(A.z, zr, A.w));
    mv[f] = M.x;
    if (A.x == 0.f) {
      if (cv[f] < -M.x) {
        hi = xl - 1;
        hash = false;
      } else if (!(cv[f] > M.x)) {
        ok = false;
      }
      continue;
    }
    float th = fminf(fmaxf(-cv[f] * M.y, (float)(xl - 1)), (float)(xh + 1));
    int kb;
    (void)ffloor_magic(th, kb);
    const int k = kb - MAGIC_BITS;
    if (A.x > 0.f) {
      if (k + 1 > lo) {
        lo = k + 1;
        Al = A.x;
        cl = cv[f];
        ml = M.x;
        hasl = true;
      }
    } else if (k < hi) {
      hi = k;
      Ah = A.x;
      ch = cv[f];
      mh = M.x;
      hash = true;
    }
  }
  if (lo <= hi) {
#pragma unroll
    for (int f = 0; f < 4; ++f)
      if (Av[f] != 0.f) ok = ok && fmaf(Av[f], (float)(Av[f] > 0.f ? lo : hi), cv[f]) > mv[f];
  }
  if (hasl && lo - 1 >= xl) ok = ok && fmaf(Al, (float)(lo - 1), cl) < -ml;
  if (hash && hi + 1 <= xh) ok = ok && fmaf(Ah, (float)(hi + 1), ch) < -mh;
  careful = !ok;
  if constexpr (!FAST) {
    if (!ok) span_careful(r, fp, xl, xh, yi, zi, lo, hi);
  }
}

// The faces of an item sorted by the sign of A.x (computed by the set-up
// kernel into the record): "low" faces (A.x > 0) bound a row from below,
// "high" faces (A.x < 0) from above, and faces with A.x == 0 (or NaN) are
// constant along a row.  order holds the face ids in that order, 2 bits
// each; shape = (number of low faces) | (number of high faces) << 4 (0x13:
// three low faces and one high face).
static __device__ __forceinline__ void face_order(const float ax[4], int& order, int& shape) {
  int lo_ids = 0, hi_ids = 0, z_ids = 0, nl = 0, nh = 0, nz = 0;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    if (ax[f] > 0.f) {
      lo_ids |= f << (2 * nl);
      ++nl;
    } else if (ax[f] < 0.f) {
      hi_ids |= f << (2 * nh);
      ++nh;
    } else {
      z_ids |= f << (2 * nz);
      ++nz;
    }
  }
  order = lo_ids | (hi_ids << (2 * nl)) | (z_ids << (2 * (nl + nh)));
  shape = nl | (nh << 4);
}

static __device__ __forceinline__ float2 lds2(const float* p) {
  float2 v;
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
  return v;
}

// row_span for an item whose faces are sorted (face_order), NL low and NH
// high faces: the same span and the same certification without tracking a
// binding face.  h = fl(A.x x + c) is non-decreasing in x for a low face and
// non-increasing for a high one, and |h - H| <= mu at every voxel of the box
// (H: the FP64 predicate), so: h(lo) > mu on every low face and h(hi) > mu on
// every high face put all of [lo, hi] inside; h(lo - 1) < -mu on some low
// face puts every voxel left of lo outside, h(hi + 1) < -mu on some high face
// every voxel right of hi.  A constant face with c < -mu empties the row.
template <int NL, int NH>
static __device__ __forceinline__ void row_span_sorted(const ItemRec& r, int order, int xl, int xh, int yi, int zi,
                                                       int& lo, int& hi, bool& careful) {
  constexpr int NF = NL + NH;
  const float yr = (float)yi, zr = (float)zi;
  const float tlo = (float)(xl - 1), thi = (float)(xh + 1);
  float A[4], c[4], m[4];
  lo = xl;
  hi = xh;
  bool ok = true, zout = false;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int f = (order >> (2 * i)) & 3;
    const float4 a = lds4(&r.fa[f][0]);
    const float2 mm = lds2(&r.fm[f][0]);
    A[i] = a.x;
    c[i] = fmaf(a.y, yr, fmaf(a.z, zr, a.w));
    m[i] = mm.x;
    if (i < NF) {
      const float th = fminf(fmaxf(-c[i] * mm.y, tlo), thi);
      int kb;
      (void)ffloor_magic(th, kb);
      if (i < NL)
        lo = max(lo, kb - (MAGIC_BITS - 1));
      else
        hi = min(hi, kb - MAGIC_BITS);
    } else {
      zout = zout || c[i] < -m[i];
      ok = ok && (c[i] > m[i] || c[i] < -m[i]);
    }
  }
  const float flo = (float)lo, fhi = (float)hi;
  if (lo <= hi) {
#pragma unroll
    for (int i = 0; i < NF; ++i) ok = ok && fmaf(A[i], i < NL ? flo : fhi, c[i]) > m[i];
  }
  if (NL > 0 && lo - 1 >= xl) {
    bool out = false;
#pragma unroll
    for (int i = 0; i < NL; ++i) out = out || fmaf(A[i], flo - 1.0f, c[i]) < -m[i];
    ok = ok && out;
  }
  if (NH > 0 && hi + 1 <= xh) {
    bool out = false;
#pragma unroll
    for (int i = NL; i < NF; ++i) out = out || fmaf(A[i], fhi + 1.0f, c[i]) < -m[i];
    ok = ok && out;
  }
  if (zout) {
    lo = xl;
    hi = xl - 1;
    ok = true;
  }
  careful = !ok;
}

// Black decision of one sample where the FP32 cell cannot decide it: FP64
// mapped coordinate (definition), its support, and the plain partner image.
static __device__ __noinline__ bool black_exact(const ItemRec& r, const DevProblem& pr, int x, int y, int z) {
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


// True when every 4x4x4 voxel block that meets the box [x0, x1] x [y0, y1] x
// [z0, z1] (inclusive, inside the image of dimensions nx, ny) holds only 0s,
// from the image's block occupancy bitmap (DevProblem::occ).
static __device__ __forceinline__ bool occ_box_zero(const unsigned long long* __restrict__ occ, int nx, int ny,
                                                    int x0, int y0, int z0, int x1, int y1, int z1) {
  const int BY = (ny + 3) >> 2, W = (((nx + 3) >> 2) + 63) >> 6;
  const int bx0 = x0 >> 2, bx1 = x1 >> 2, w0 = bx0 >> 6, w1 = bx1 >> 6;
  for (int bz = z0 >> 2; bz <= (z1 >> 2); ++bz)
    for (int by = y0 >> 2; by <= (y1 >> 2); ++by) {
      const unsigned long long* row = occ + ((long)bz * BY + by) * W;
      for (int w = w0; w <= w1; ++w) {
        const int lo = w == w0 ? (bx0 & 63) : 0, hi = w == w1 ? (bx1 & 63) : 63;
        if (__ldg(row + w) & (~0ull >> (63 - hi)) & (~0ull << lo)) return false;
      }
    }
  return true;
}

// True when the 4x4x4 blocks bx0..bx1 of block row (by, bz) of a bitmap
// (DevProblem::occ layout, BY = ceil(ny / 4), W words per block row) are
// all clear; one word, or two where the range crosses a word.
static __device__ __forceinline__ bool occ_blocks_clear(const unsigned long long* __restrict__ occ, int BY, int W,
                                                        int bx0, int bx1, int by, int bz) {
  const unsigned long long* row = occ + ((long)bz * BY + by) * W;
  const int w0 = bx0 >> 6, w1 = bx1 >> 6;
  if (w0 == w1) return !(__ldg(row + w0) & (~0ull >> (63 - (bx1 & 63))) & (~0ull << (bx0 & 63)));
  if (__ldg(row + w0) & (~0ull << (bx0 & 63))) return false;
  for (int w = w0 + 1; w < w1; ++w)
    if (__ldg(row + w)) return false;
  return !(__ldg(row + w1) & (~0ull >> (63 - (bx1 & 63))));
}

// ------------------------------------------------------------ raster + sample
struct WarpSmem {
  ItemRec rec;
  int2 meta[32];     // (exclusive voxel prefix, own plain index of x0) per row
  float4 pr0[32];    // mapped partner-relative coordinate of x0 per row
  // empty-space test of the rows: own and partner block occupancy bitmaps,
  // partner dimensions, mode (0 off, 1 own rows only: the partner region is
  // all 0, 2 own rows and the partner region)
  const unsigned long long* zown;
  const unsigned long long* zpar;
  int zn[3];
  int zon;
  unsigned execd;  // samples of the current item mapped and sampled so far
  int pend;        // fast pass: the second item of lane 0's last claimed pair, or -1
  // loop state parked here while the voxel loop runs (it holds no registers
  // there): per slice lane the first row index and first y of its slice, the
  // slice group, the batch, the rows of the group, the own image's nx and ny
  int yex[32], ylos[32];
  int zb, R, nxo, nyo;
};

template <int ST>
struct Cell {
  float4 a, b;  // ST_F32: 8 corners
};
template <>
struct Cell<ST_BF16> {
  uint4 w;
};
template <>
struct Cell<ST_F16> {
  uint4 w;
};

template <int ST>
static __device__ __forceinline__ void cell_load(const void* cells, unsigned idx, Cell<ST>& c) {
  if constexpr (ST == ST_F32) {
    const float4* p = (const float4*)cells + 2 * (size_t)idx;
    c.a = __ldg(p);
    c.b = __ldg(p + 1);
  } else {
    c.w = __ldg((const uint4*)cells + idx);
  }
}

template <int ST>
static __device__ __forceinline__ float cell_interp(const Cell<ST>& c, float fx, float fy, float fz) {
  float c0, c1, c2, c3, c4, c5, c6, c7;
  if constexpr (ST == ST_F32) {
    // f32 cells hold (c0, c1 - c0, c2, c3 - c2, c4, c5 - c4, c6, c7 - c6): the
    // same FP32 differences the first level would form, one FMA each
    const float a0 = fmaf(fx, c.a.y, c.a.x);
    const float a1 = fmaf(fx, c.a.w, c.a.z);
    const float a2 = fmaf(fx, c.b.y, c.b.x);
    const float a3 = fmaf(fx, c.b.w, c.b.z);
    const float b0 = fmaf(fy, a1 - a0, a0);
    const float b1 = fmaf(fy, a3 - a2, a2);
    return fmaf(fz, b1 - b0, b0);
  } else if constexpr (ST == ST_BF16) {
    c0 = bf16lo(c.w.x); c1 = bf16hi(c.w.x); c2 = bf16lo(c.w.y); c3 = bf16hi(c.w.y);
    c4 = bf16lo(c.w.z); c5 = bf16hi(c.w.z); c6 = bf16lo(c.w.w); c7 = bf16hi(c.w.w);
  } else {
    c0 = f16lo(c.w.x); c1 = f16hi(c.w.x); c2 = f16lo(c.w.y); c3 = f16hi(c.w.y);
    c4 = f16lo(c.w.z); c5 = f16hi(c.w.z); c6 = f16lo(c.w.w); c7 = f16hi(c.w.w);
  }
  float a0 = fmaf(fx, c1 - c0, c0);
  float a1 = fmaf(fx, c3 - c2, c2);
  float a2 = fmaf(fx, c5 - c4, c4);
  float a3 = fmaf(fx, c7 - c6, c6);
  float b0 = fmaf(fy, a1 - a0, a0);
  float b1 = fmaf(fy, a3 - a2, a2);
  return fmaf(fz, b1 - b0, b0);
}

// Black decision of a sample whose FP32 fraction is within delta of 0 or 1
// on some axis, from the zero mask of the 4x4x4 block around its cell.  Per
// axis the true support is {i, i+1} unless the fraction is near 0 (then
// {i-1, i}, {i} or {i, i+1}) or near 1 ({i, i+1}, {i+1} or {i+1, i+2}).
// Black for certain if the union of the possible supports is all 0; not
// black for certain if their intersection holds a nonzero voxel.  Returns
// 1 / 0, or -1 when the FP64 definition must decide.
static __device__ __forceinline__ int black_near(unsigned long long zm, float fx, float fy, float fz, float delta) {
  // 4-bit sets over the offsets -1..2 (bit 0 = offset -1)
  auto axis = [&](float f, unsigned& un, unsigned& in) {
    if (f <= delta) {
      un = 0x7u;
      in = 0x2u;
    } else if (f >= 1.0f - delta) {
      un = 0xEu;
      in = 0x4u;
    } else {
      un = in = 0x6u;
    }
  };
  unsigned ux, ix, uy, iy, uz, iz;
  axis(fx, ux, ix);
  axis(fy, uy, iy);
  axis(fz, uz, iz);
  auto box = [](unsigned mx, unsigned my, unsigned mz) {
    // rows of 4 bits: (y, z) -> bits 4 y + 16 z
    unsigned long long row = 0ull;
    for (int y = 0; y < 4; ++y)
      if ((my >> y) & 1u) row |= (unsigned long long)mx << (4 * y);
    unsigned long long m = 0ull;
    for (int z = 0; z < 4; ++z)
      if ((mz >> z) & 1u) m |= row << (16 * z);
    return m;
  };
  const unsigned long long U = box(ux, uy, uz), I = box(ix, iy, iz);
  if ((zm & U) == U) return 1;
  if ((zm & I) != I) return 0;
  return -1;
}

// Cell flags (built with the corner cells): bit0 some corner is 0, bit1 all
// corners are 0, bit2 every voxel of the 4x4x4 block around the cell is 0,
// bit3 no voxel of that block is 0, bit4 = bit0 and neither bit2 nor bit3.
// The exact support of a sample always lies inside that block, so bits 2/3
// settle the black test outright (bit2 implies bit1, bit3 rules out bit1);
// a cell with no 0 corner is never black (every support shares a corner
// with the FP32 cell).  So the test is bit1, except where bit4 is set and
// the sample lies near a cell face.
enum { CF_ANY0 = 1, CF_ALL0 = 2, CF_NB_ALL0 = 4, CF_NB_NONE0 = 8, CF_NEAR = 16 };

// Threads per SM the register budget is sized for (2048 / 1024 / 768 / 512).
#ifndef DMR_RASTER_THREADS_PER_SM
#define DMR_RASTER_THREADS_PER_SM 768
#endif

// Two kernels share this body.  FAST = true: no function calls in the row
// and voxel loops (a call there costs ~60 registers per thread, a third of
// the SM's resident warps); an item with a row whose span the margins cannot
// certify, or a sample whose black decision needs the FP64 definition, is
// abandoned and appended to b.slow.  FAST = false: the same item logic with
// the careful span and the exact black decision inline, over the items of
// b.slow: with few such items the warps of a CTA share each item, with many
// one warp takes an item as in the fast pass.  Which items are handed over
// (and so the mode) depends only on the data, so results do not depend on
// the tile shape.
template <int ST, int WARPS, int VPL, bool FAST>
__global__ void __launch_bounds__(WARPS * 32, (FAST && DMR_RASTER_THREADS_PER_SM / (WARPS * 32) > 0
                                                    ? DMR_RASTER_THREADS_PER_SM / (WARPS * 32)
                                                    : (FAST ? 1 : 6)))
    k_raster(const DevProblem* __restrict__ probs, Batch b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WarpSmem* ws = (WarpSmem*)smem_raw + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  const unsigned lemask = 0xffffffffu >> (31 - lane);
  const int n_items = 2 * b.n_tt;
  // full-logic pass: one warp per item when the handed-over items outnumber
  // the grid's warps, else the WARPS warps of a CTA share an item (row
  // batches dealt round-robin, partial sums added in warp order); uniform
  // over the grid
  __shared__ int s_item;
  __shared__ double s_part[WARPS];
  __shared__ int s_cov[WARPS];
  const bool cta_mode = !FAST && WARPS > 1 && *(volatile unsigned*)(b.work + 1) < gridDim.x * (unsigned)WARPS;
  const int rstep = cta_mode ? 32 * WARPS : 32;
  // fast pass: lane 0 claims items two at a time (one atomic per pair); the
  // second waits in shared memory
  if (FAST && lane == 0) ws->pend = -1;
  for (;;) {
    int item = 0;
    if (cta_mode) {
      if (threadIdx.x == 0) {
        const unsigned w = atomicAdd(b.work + 2, 1u);
        s_item = w < *(volatile unsigned*)(b.work + 1) ? b.slow[w] : n_items;
      }
      __syncthreads();
      item = s_item;
    } else {
      if (lane == 0) {
        if constexpr (FAST) {
          const int pend = *(volatile int*)&ws->pend;
          if (pend >= 0) {
            item = pend;
            ws->pend = -1;
          } else {
            item = (int)atomicAdd(b.work, 2u);
            ws->pend = item + 1;
          }
        } else {
          const unsigned w = atomicAdd(b.work + 2, 1u);
          item = w < *(volatile unsigned*)(b.work + 1) ? b.slow[w] : n_items;
        }
      }
      item = __shfl_sync(FULL_MASK, item, 0);
    }
    if (item >= n_items) break;
    constexpr int NW = sizeof(ItemRec) / 16;
    WarpSmem* rs = cta_mode ? (WarpSmem*)smem_raw : ws;  // whose record the warp reads
    if (cta_mode) {
      const int4* src = (const int4*)(b.rec + item);
      int4* dst = (int4*)&rs->rec;
      for (int i = threadIdx.x; i < NW; i += 32 * WARPS) dst[i] = __ldg(src + i);
      __syncthreads();
    } else {
      // the fast pass reads a record only up to its FP64 vertex copies (those
      // serve the careful spans and the exact black decision of the
      // full-logic pass), so it copies only those words
      constexpr int NR = FAST ? (int)(offsetof(ItemRec, X) / 16) : NW;
      const int4* src = (const int4*)(b.rec + item);
      int4* dst = (int4*)&ws->rec;
      for (int i = lane; i < NR; i += 32) dst[i] = __ldg(src + i);
      __syncwarp();
    }
    const ItemRec& r = rs->rec;
    float sum = 0.f, comp = 0.f;
    int cov = 0;
    bool need_exact = false;  // FAST: some sample needs the FP64 black decision
    if (r.flags & 1) {
      const DevProblem& pr = probs[r.prob];
      const int d = r.dir;
      const uint32_t fp = pr.fperm[r.tet];
      const void* own_img = pr.plain[d];
      const void* cells = pr.cells[1 - d];
      const uint8_t* cflag = pr.cflag[1 - d];
      const unsigned long long* cmask = pr.cmask[1 - d];
      const unsigned Sy = (unsigned)(pr.n[1 - d][0] + 2), Sz = (unsigned)(pr.n[1 - d][1] + 2) * Sy;
      const bool black = pr.black_rule != 0;
      const bool pzero = (r.flags & 4) != 0;
      // cell flags are read only where a sample may be black
      const bool cfload = black && !(r.flags & 8);
      // empty-space test per row: a row whose own voxels are all 0 and whose
      // samples can reach only partner voxels that are 0 adds exactly 0
      // (every sample is 0 and black: black against black, or 0 - 0), so it
      // is counted but not sampled.  Needs a finite small map (bit5) and a
      // partner region that is not known to hold no 0 (bit3);
      // it reads the images' 4x4x4 block occupancy bitmaps (a few KB, cached
      // on chip).  Its parameters wait in shared memory (read where used, so
      // that they hold no registers across the loops).
      if (lane == 0) {
        const unsigned long long* zo = pr.occ[d];
        const unsigned long long* zp = pr.occd[1 - d];
        const bool on = zo != nullptr && zp != nullptr && (r.flags & 32) && !(r.flags & 8);
        ws->zown = zo;
        ws->zpar = zp;
        ws->zon = on ? (pzero ? 1 : 2) : 0;
        for (int a = 0; a < 3; ++a) ws->zn[a] = pr.n[1 - d][a];
        ws->execd = 0u;
        ws->nxo = pr.n[d][0];
        ws->nyo = pr.n[d][1];
      }
      __syncwarp();
      // the record's integer fields, read where used
#define RV(f) (*(volatile int*)&(f))
      for (int zb = r.b0[2]; zb <= RV(r.b1[2]); zb = RV(ws->zb) + 32) {
        const int z = zb + lane;
        const int Oy = RV(r.O[1]);
        int ycnt = 0, ylo = 0;
        if (z <= RV(r.b1[2])) {
          float ylf, yhf;
          slice_yrange(r, (float)(z - RV(r.O[2])), ylf, yhf);
          float slack = 1.0f / 256.0f + 1e-5f * fabsf(yhf);
          int y0 = max(RV(r.b0[1]), (int)ceilf(ylf - slack) + Oy);
          int y1 = min(RV(r.b1[1]), (int)floorf(yhf + slack) + Oy);
          if (ylf <= yhf && y1 >= y0) {
            ylo = y0;
            ycnt = y1 - y0 + 1;
          }
        }
        const int yincl = warp_incl_scan(ycnt, lane);
        ws->yex[lane] = yincl - ycnt;
        ws->ylos[lane] = ylo;
        ws->zb = zb;  // every lane stores the same value
        if (lane == 31) ws->R = yincl;
        __syncwarp();
        for (int rb = cta_mode ? 32 * wid : 0; rb < RV(ws->R); rb += rstep) {
          const int R = RV(ws->R);
          const int rr = rb + lane;
          const bool has_row = rr < R;
          const int rq = has_row ? rr : R - 1;
          int s = 0;
#pragma unroll
          for (int step = 16; step > 0; step >>= 1) {
            const int cs = s + step;
            const int e = RV(ws->yex[cs & 31]);
            if (cs < 32 && e <= rq) s = cs;
          }
          const int e_s = RV(ws->yex[s]);
          const int yl_s = RV(ws->ylos[s]);
          const int zrow = RV(ws->zb) + s;
          const int yrow = yl_s + (rq - e_s);
          const int Ox = RV(r.O[0]);
          const int xl = RV(r.b0[0]) - Ox, xh = RV(r.b1[0]) - Ox;
          const int nxo = RV(ws->nxo), nyo = RV(ws->nyo);
          int xcnt = 0, x0 = 0;
          bool careful = false;
          if (has_row) {
            const int Oy = RV(r.O[1]), Oz = RV(r.O[2]);
            const uint32_t fp = pr.fperm[RV(r.tet)];
            int lo, hi;
            const int yi = yrow - Oy, zi = zrow - Oz;
            if constexpr (FAST) {
              const int forder = *(volatile int*)&r.forder;
              switch (*(volatile int*)&r.fshape) {
                case 0x13: row_span_sorted<3, 1>(r, forder, xl, xh, yi, zi, lo, hi, careful); break;
                case 0x22: row_span_sorted<2, 2>(r, forder, xl, xh, yi, zi, lo, hi, careful); break;
                case 0x31: row_span_sorted<1, 3>(r, forder, xl, xh, yi, zi, lo, hi, careful); break;
                case 0x12: row_span_sorted<2, 1>(r, forder, xl, xh, yi, zi, lo, hi, careful); break;
                case 0x21: row_span_sorted<1, 2>(r, forder, xl, xh, yi, zi, lo, hi, careful); break;
                case 0x11: row_span_sorted<1, 1>(r, forder, xl, xh, yi, zi, lo, hi, careful); break;
                default: row_span<true>(r, fp, xl, xh, yi, zi, lo, hi, careful);
              }
            } else {
              row_span<false>(r, fp, xl, xh, yi, zi, lo, hi, careful);
            }
            if (hi >= lo) {
              xcnt = hi - lo + 1;
              x0 = lo + Ox;
            }
          }
          if constexpr (FAST) {
            if (__any_sync(FULL_MASK, careful)) goto handover;
          }
          // every voxel of the batch's rows is one sample (counted)
          cov += __reduce_add_sync(FULL_MASK, (unsigned)xcnt);
          if ((*(volatile int*)&r.flags & 20) == 20) {
            // own and partner voxels all 0: every sample adds 0, only the
            // batch's voxel count matters
            continue;
          }
          int xs = xcnt;  // voxels of this row that are sampled
          if (xcnt > 0 && *(volatile int*)&ws->zon) {
            bool skip = occ_blocks_clear(*(const unsigned long long* volatile*)&ws->zown, (nyo + 3) >> 2,
                                         (((nxo + 3) >> 2) + 63) >> 6, x0 >> 2, (x0 + xcnt - 1) >> 2, yrow >> 2,
                                         zrow >> 2);
            if (skip && *(volatile int*)&ws->zon == 2) {
              // the samples' FP32 positions run from the row start p to
              // p + (xcnt - 1) gx (the loop's own expressions, monotone in the
              // step, clamps included)
              const float vx = (float)(x0 - Ox), vy = (float)(yrow - RV(r.O[1])), vz = (float)(zrow - RV(r.O[2]));
              const float4 g0 = lds4(&r.G[0][0]), g1 = lds4(&r.G[1][0]), g2 = lds4(&r.G[2][0]);
              const float4 gx = lds4(&r.gx[0]), lo = lds4(&r.clo[0]), hi = lds4(&r.chi[0]);
              const float dl = (float)(xcnt - 1);
              float ax = vx + fmaf(g0.x, vx, fmaf(g0.y, vy, fmaf(g0.z, vz, g0.w)));
              float ay = vy + fmaf(g1.x, vx, fmaf(g1.y, vy, fmaf(g1.z, vz, g1.w)));
              float az = vz + fmaf(g2.x, vx, fmaf(g2.y, vy, fmaf(g2.z, vz, g2.w)));
              float qx = fmaf(dl, gx.x, ax), qy = fmaf(dl, gx.y, ay), qz = fmaf(dl, gx.z, az);
              if (!(*(volatile int*)&r.flags & 2)) {
                ax = fminf(fmaxf(ax, lo.x), hi.x);
                ay = fminf(fmaxf(ay, lo.y), hi.y);
                az = fminf(fmaxf(az, lo.z), hi.z);
                qx = fminf(fmaxf(qx, lo.x), hi.x);
                qy = fminf(fmaxf(qy, lo.y), hi.y);
                qz = fminf(fmaxf(qz, lo.z), hi.z);
              }
              // blocks holding the samples' FP32 positions, against the
              // partner bitmap dilated by one block: a sample's exact support
              // and FP32 cell lie within 1 voxel below / 2 above its position,
              // inside the block around the position's block
              int zn[3];
              for (int a = 0; a < 3; ++a) zn[a] = *(volatile int*)&ws->zn[a];
              // (block indices clamped to the image's blocks, as the supports
              // are clamped to the image)
              auto blk = [](float v, int o, int n) { return min(max(((int)floorf(v) + o) >> 2, 0), (n - 1) >> 2); };
              const int lx = blk(fminf(ax, qx), *(volatile int*)&r.Op[0], zn[0]);
              const int ly = blk(fminf(ay, qy), *(volatile int*)&r.Op[1], zn[1]);
              const int lz = blk(fminf(az, qz), *(volatile int*)&r.Op[2], zn[2]);
              const int hx = blk(fmaxf(ax, qx), *(volatile int*)&r.Op[0], zn[0]);
              const int hy = blk(fmaxf(ay, qy), *(volatile int*)&r.Op[1], zn[1]);
              const int hz = blk(fmaxf(az, qz), *(volatile int*)&r.Op[2], zn[2]);
              const int BY = (zn[1] + 3) >> 2, W = (((zn[0] + 3) >> 2) + 63) >> 6;
              const unsigned long long* zp = *(const unsigned long long* volatile*)&ws->zpar;
              for (int bz = lz; bz <= hz && skip; ++bz)
                for (int by = ly; by <= hy && skip; ++by) skip = occ_blocks_clear(zp, BY, W, lx, hx, by, bz);
            }
            if (skip) xs = 0;
          }
          const unsigned nzm = __ballot_sync(FULL_MASK, xs > 0);
          const int cidx = __popc(nzm & (lemask >> 1));
          const int xincl = warp_incl_scan(xs, lane);
          const int xexcl = xincl - xs;
          const int T = __shfl_sync(FULL_MASK, xincl, 31);
          if (T == 0) continue;
          if (xs > 0) {
            const float vx = (float)(x0 - Ox), vy = (float)(yrow - RV(r.O[1])), vz = (float)(zrow - RV(r.O[2]));
            const float4 g0 = lds4(&r.G[0][0]), g1 = lds4(&r.G[1][0]), g2 = lds4(&r.G[2][0]);
            const float px = vx + fmaf(g0.x, vx, fmaf(g0.y, vy, fmaf(g0.z, vz, g0.w)));
            const float py = vy + fmaf(g1.x, vx, fmaf(g1.y, vy, fmaf(g1.z, vz, g1.w)));
            const float pz = vz + fmaf(g2.x, vx, fmaf(g2.y, vy, fmaf(g2.z, vz, g2.w)));
            ws->meta[cidx] = make_int2(xexcl, (zrow * nyo + yrow) * nxo + x0);
            ws->pr0[cidx] = make_float4(px, py, pz, 0.f);
          }
          __syncwarp();
          const float gxx = r.gx[0], gxy = r.gx[1], gxz = r.gx[2], delta = r.gx[3];
          const float clx = r.clo[0], cly = r.clo[1], clz = r.clo[2];
          const float chx = r.chi[0], chy = r.chi[1], chz = r.chi[2];
          const unsigned cbase = r.cbase;
          // partner tet well inside the image and a small map: mapped
          // coordinates cannot leave [-1, n], so the clamps are skipped
          const bool inside = (r.flags & 2) != 0;
          if (lane == 0 && !pzero) ws->execd += (unsigned)T;
          int rows_before = 0;
          // plain FP32 partial sum over at most 256 voxels of the batch (<= 8
          // samples per lane), folded into the Kahan pair afterwards; the
          // fold points do not depend on the tile shape
          float bsum = 0.f;
          if (pzero) {
            // every partner voxel these samples can reach is 0: each sample is
            // 0 and black, so only the own image is read (items whose own
            // voxels are all 0 as well never get here).  Same per-lane order
            // and fold points as the loop below (identical sums).
            for (int vb = 0; vb < T; vb += 32) {
              if (vb != 0 && (vb & 255) == 0) {
                const float yk = bsum - comp;
                const float tk = sum + yk;
                comp = (tk - sum) - yk;
                sum = tk;
                bsum = 0.f;
              }
              const unsigned bit = (xs > 0 && xexcl >= vb && xexcl < vb + 32) ? (1u << (xexcl - vb)) : 0u;
              const unsigned sm = __reduce_or_sync(FULL_MASK, bit);
              const int row = rows_before + __popc(sm & lemask) - 1;
              rows_before += __popc(sm);
              if (vb + lane < T) {
                const int2 mt = ws->meta[row];
                const float o = load_plain<ST>(own_img, mt.y + (vb + lane - mt.x));
                bsum += black ? (o != 0.0f ? 1.0f : 0.0f) : o * o;
              }
            }
          } else
          for (int vb = 0; vb < T; vb += 32 * VPL) {
            if (vb != 0 && (vb & 255) == 0) {
              const float yk = bsum - comp;
              const float tk = sum + yk;
              comp = (tk - sum) - yk;
              sum = tk;
              bsum = 0.f;
            }
            int row[VPL], vv[VPL];
#pragma unroll
            for (int u = 0; u < VPL; ++u) {
              const int wb = vb + 32 * u;
              const unsigned bit = (xs > 0 && xexcl >= wb && xexcl < wb + 32) ? (1u << (xexcl - wb)) : 0u;
              const unsigned sm = __reduce_or_sync(FULL_MASK, bit);
              row[u] = rows_before + __popc(sm & lemask) - 1;
              rows_before += __popc(sm);
              vv[u] = wb + lane;
            }
            // stage A: addresses and loads of all VPL voxels
            Cell<ST> cell[VPL];
            float own[VPL], fx[VPL], fy[VPL], fz[VPL];
            uint8_t cf[VPL];
            int oi[VPL];
            unsigned cix[VPL];
#pragma unroll
            for (int u = 0; u < VPL; ++u) {
              if (vv[u] < T) {
                const int2 mt = ws->meta[row[u]];
                const float4 p0 = ws->pr0[row[u]];
                const int dx = vv[u] - mt.x;
                const float dxf = __int_as_float(dx + MAGIC_BITS) - MAGIC;
                float px = fmaf(dxf, gxx, p0.x), py = fmaf(dxf, gxy, p0.y), pz = fmaf(dxf, gxz, p0.z);
                if (!inside) {
                  px = fminf(fmaxf(px, clx), chx);
                  py = fminf(fmaxf(py, cly), chy);
                  pz = fminf(fmaxf(pz, clz), chz);
                }
                int ix, iy, iz;
                const float flx = ffloor_magic(px, ix), fly = ffloor_magic(py, iy), flz = ffloor_magic(pz, iz);
                fx[u] = px - flx;
                fy[u] = py - fly;
                fz[u] = pz - flz;
                const unsigned ci = cbase + (unsigned)iz * Sz + (unsigned)iy * Sy + (unsigned)ix;
                cix[u] = ci;
                oi[u] = mt.y + dx;
                cell_load<ST>(cells, ci, cell[u]);
                own[u] = load_plain<ST>(own_img, oi[u]);
                cf[u] = cfload ? __ldg(cflag + ci) : (uint8_t)0;
              }
            }
            // stage B: interpolate, compare, accumulate
#pragma unroll
            for (int u = 0; u < VPL; ++u) {
              if (vv[u] < T) {
                const float s = cell_interp<ST>(cell[u], fx[u], fy[u], fz[u]);
                const float o = own[u];
                const float dd = o - s;
                float d2 = dd * dd;
                if (black) {
                  const unsigned f = cf[u];
                  bool blk = (f & CF_ALL0) != 0;
                  if (f & CF_NEAR) {
                    const bool nearp = fminf(fminf(fx[u], fy[u]), fz[u]) <= delta ||
                                       fmaxf(fmaxf(fx[u], fy[u]), fz[u]) >= 1.0f - delta;
                    if (nearp) {
                      const int dec = black_near(__ldg(cmask + cix[u]), fx[u], fy[u], fz[u], delta);
                      if (dec >= 0) {
                        blk = dec != 0;
                      } else if constexpr (FAST) {
                        need_exact = true;
                        blk = false;
                      } else {
                        const int xa = oi[u] % nxo;
                        const int rem = oi[u] / nxo;
                        blk = black_exact(r, pr, xa, rem % nyo, rem / nyo);
                      }
                    }
                  }
                  if ((o == 0.0f) != blk) d2 = 1.0f;
                }
                bsum += d2;
              }
            }
            if constexpr (FAST) {
              if (__any_sync(FULL_MASK, need_exact)) goto handover;
            }
          }
          {
            const float yk = bsum - comp;
            const float tk = sum + yk;
            comp = (tk - sum) - yk;
            sum = tk;
          }
          __syncwarp();
        }
      }
    }
    {
      // error-free warp reduction of (sum, -comp)
      float hi = sum, lo = -comp;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(FULL_MASK, hi, o);
        const float ol = __shfl_xor_sync(FULL_MASK, lo, o);
        const float sh = hi + oh;
        const float bb = sh - hi;
        const float err = (hi - (sh - bb)) + (oh - bb);
        hi = sh;
        lo = lo + ol + err;
      }
      const int covt = __shfl_sync(FULL_MASK, cov, 0);  // cov is warp-uniform
      if (lane == 0 && (rs->rec.flags & 1) && ws->execd)
        atomicAdd(probs[rs->rec.prob].executed, (unsigned long long)ws->execd);
      if (!cta_mode) {
        if (lane == 0) {
          b.o_ssd[item] = (double)hi + (double)lo;
          b.o_cov[item] = covt;
        }
        __syncwarp();
      } else {
        if (lane == 0) {
          s_part[wid] = (double)hi + (double)lo;
          s_cov[wid] = covt;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          double t = 0.0;
          int c = 0;
          for (int w = 0; w < WARPS; ++w) {
            t += s_part[w];
            c += s_cov[w];
          }
          b.o_ssd[item] = t;
          b.o_cov[item] = c;
        }
        __syncthreads();
      }
    }
    continue;
  handover:
    // FAST only: the item goes to the full-logic kernel, which writes its outputs
    if (lane == 0) b.slow[atomicAdd(b.work + 1, 1u)] = item;
    __syncwarp();
  }
}

template <int ST, int WARPS, int VPL, bool FAST>
static void raster_launch_one(const DevProblem* probs, const Batch& b, int n_sm, cudaStream_t st) {
  const int threads = 32 * WARPS;
  const size_t smem = sizeof(WarpSmem) * WARPS;
  const long items = 2L * b.n_tt;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_raster<ST, WARPS, VPL, FAST>, threads, smem);
  if (per_sm < 1) per_sm = 1;
  long blocks = (long)n_sm * per_sm;
  const long need = (items + WARPS - 1) / WARPS;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  k_raster<ST, WARPS, VPL, FAST><<<(unsigned)blocks, threads, smem, st>>>(probs, b);
}

// The fast kernel with the requested tile shape, then the full-logic kernel
// over the items it handed over (a persistent grid that exits at once when
// there are none).
template <int ST>
static void raster_launch(const DevProblem* probs, const Batch& b, int warps, int vpw, int n_sm, cudaStream_t st,
                          cudaStream_t side, cudaEvent_t fork) {
  const int vpl = vpw >= 128 ? 4 : (vpw >= 64 ? 2 : 1);
  bool done = false;
  if (side && fork) {
    cudaEventRecord(fork, st);
    cudaStreamWaitEvent(side, fork, 0);
  }
#define DMR_RL(W, V)                                          \
  if (!done && warps == W && vpl == V) {                      \
    raster_launch_one<ST, W, V, true>(probs, b, n_sm, st);    \
    done = true;                                              \
  }
  DMR_RL(4, 1) DMR_RL(4, 2) DMR_RL(4, 4)
  DMR_RL(8, 1) DMR_RL(8, 2) DMR_RL(8, 4)
  DMR_RL(16, 1) DMR_RL(16, 2) DMR_RL(16, 4)
#undef DMR_RL
  if (!done) raster_launch_one<ST, 4, 1, true>(probs, b, n_sm, st);
  raster_launch_one<ST, 4, 1, false>(probs, b, n_sm, st);
}

}  // namespace dmr
