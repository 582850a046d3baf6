/*
 * dmr_oracle.c -- plain, slow FP64 CPU oracle for the objectives of
 * multi-objective dual simplex-mesh deformable registration
 * (Andreadis, Bosman, Alderliesten, arXiv 2202.11001).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this file.  It shares no code, header,
 * table or helper with the CUDA library; each side implements the same
 * written definitions on its own.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared -fopenmp.  FMA contraction
 * must stay off: every FP64 expression below is a decision-carrying
 * definition (inside test, fold test, mapped black-rule coordinate) and is
 * evaluated with one rounding per written operation, in the written order.
 *
 * What it computes, with the paper passage each piece follows:
 *  - Sec. 2.1, Fig. 1A/1B: a lattice of m_x*m_y*m_z points; every cube of 8
 *    points is cut into 6 tetrahedra along one main diagonal, and the
 *    diagonal is mirrored between neighbouring cubes (2x2x2 cube groups).
 *    Reading: the diagonal of cube (cx,cy,cz) joins its all-even corner to
 *    its all-odd corner; the 6 tets are the 6 axis-order paths along it.
 *  - Sec. 2.1: two meshes with the same topology (source mesh on the source
 *    image, target mesh on the target image); tet t of one corresponds to
 *    tet t of the other.
 *  - Sec. 2.3.1: dissimilarity = squared intensity difference of
 *    corresponding voxels, forward (source voxels mapped into the target)
 *    plus backward, a black-vs-grey mismatch costs 1, normalised by the
 *    total voxel count.  Voxels of a tet are found by rasterising it; the
 *    "top-left" tie rule is read in 3-D as: a voxel on a shared face goes to
 *    the tet on the side the face's normal lexicographically points into.
 *  - Sec. 2.3.2: deformation = Hooke springs on the 6 edges plus 4 spokes
 *    (vertex to opposite-face centroid) per tet, normalised by the edge
 *    count (SPRING); a linear-elastic energy from the deformation gradient
 *    with Lame lambda, mu is the second, flag-selected model (LINEAR).
 *  - Sec. 2.3.3: guidance = symmetric squared distance of annotated point
 *    pairs carried through the transformation, normalised by point count.
 *  - Sec. 2.3.4: folding is forbidden; counted here by signed volume plus
 *    the border-plane rule for border points.
 *  - Sec. 2.2, 2.3: every objective is a sum of per-tet (and per-landmark)
 *    terms, so a change of a point group re-evaluates only the tets that
 *    touch it (partial evaluation).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define DMO_SPRING 0
#define DMO_LINEAR 1

typedef struct {
  double ssd[2]; /* [0] forward (source voxels), [1] backward (target voxels) */
  int32_t cov[2];
  double def;
  int32_t fold;
} dmo_term;

typedef struct {
  int n[2][3];
  double sp[2][3];
  double* img[2]; /* [nz][ny][nx], owned copies */
  long nvox[2];
  int m[3];
  int P, ntet;
  int32_t* tet;       /* [ntet][4] point ids, positive rest orientation */
  int8_t* fperm;      /* [ntet][4][4]: local idx of (a,b,c) canonical, then sign */
  int32_t* star_ptr;  /* [P+1] */
  int32_t* star;      /* [4*ntet] tets per point, ascending */
  uint8_t* fixmask;   /* [P] bit a set: axis a fixed (border) */
  double* rest[2];    /* [3][P] rest coordinates per mesh */
  double* rest_vol;   /* [ntet] rest volume (mm^3) of the source mesh */
  double rest_vol_sum;
  int black_rule, model;
  double lam, mu;
  int ng;
  double* guide; /* [ng][2][3] */
  /* population state */
  int C;
  double* coords; /* [C][2][3][P] */
  dmo_term* terms; /* [C][ntet] */
  int32_t* gset;   /* [ng] guidance set of each pair (Sec. 2.3.3); NULL: each pair its own set */
  int32_t* loc;    /* [C][2][ng] */
  double* gterm;   /* [C][2][ng] */
  double* sums;    /* [C][4] raw sums */
  /* last partial evaluation */
  int ntr;
  int32_t* tr_cand;
  int32_t* tr_tptr;  /* [ntr+1] */
  int32_t* tr_tets;  /* touched tets, ascending per trial (capacity offsets tr_tptr) */
  int32_t* tr_ntt;   /* [ntr] touched-set sizes */
  dmo_term* tr_terms;
  int32_t* tr_gpt_ptr; /* [ntr+1] */
  int32_t* tr_gpts;
  double* tr_coords; /* per trial [2][3][npts] at offset 6*gptr */
  int32_t* tr_loc;   /* [ntr][2][ng] */
  double* tr_gterm;  /* [ntr][2][ng] */
  int32_t* tr_aff;   /* [ntr][2][ng] 1 if landmark re-evaluated */
  double* tr_raw;    /* [ntr][4] */
} dmo_problem;

static int g_threads = 1;

void dmo_set_threads(int n) { g_threads = n > 0 ? n : 1; }
int dmo_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---------------------------------------------------------------- topology */

static const int AXIS_ORDER[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2},
                                     {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

static int point_id(const int m[3], int a, int b, int c) {
  return a + m[0] * (b + m[1] * c);
}

int dmo_num_tets(const int* m) {
  if (m[0] < 2 || m[1] < 2 || m[2] < 2) return 0;
  return 6 * (m[0] - 1) * (m[1] - 1) * (m[2] - 1);
}

/* Sec. 2.1 / Fig. 1A-B: 6 tets per cube, diagonal mirrored per cube parity. */
void dmo_build_tets(const int* m, int32_t* tets) {
  int t = 0;
  for (int cz = 0; cz < m[2] - 1; ++cz)
    for (int cy = 0; cy < m[1] - 1; ++cy)
      for (int cx = 0; cx < m[0] - 1; ++cx) {
        int cube[3] = {cx, cy, cz};
        int start[3], dir[3];
        for (int k = 0; k < 3; ++k) {
          int par = cube[k] & 1;
          start[k] = cube[k] + par; /* the corner with even global index */
          dir[k] = par ? -1 : 1;
        }
        for (int q = 0; q < 6; ++q) {
          int v[4][3];
          for (int k = 0; k < 3; ++k) v[0][k] = start[k];
          for (int s = 0; s < 3; ++s) {
            for (int k = 0; k < 3; ++k) v[s + 1][k] = v[s][k];
            int ax = AXIS_ORDER[q][s];
            v[s + 1][ax] += dir[ax];
          }
          long e[3][3];
          for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) e[i][k] = v[i + 1][k] - v[0][k];
          long det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) +
                     e[0][1] * (e[1][2] * e[2][0] - e[1][0] * e[2][2]) +
                     e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
          int32_t id[4];
          for (int i = 0; i < 4; ++i) id[i] = point_id(m, v[i][0], v[i][1], v[i][2]);
          if (det < 0) {
            int32_t tmp = id[1];
            id[1] = id[2];
            id[2] = tmp;
          }
          for (int i = 0; i < 4; ++i) tets[4 * t + i] = id[i];
          ++t;
        }
      }
}

static int perm_parity(const int p[4]) {
  int inv = 0;
  for (int i = 0; i < 4; ++i)
    for (int j = i + 1; j < 4; ++j)
      if (p[i] > p[j]) ++inv;
  return (inv & 1) ? -1 : 1;
}

/* ------------------------------------------------------------ FP64 geometry */

static void cross3(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + (a[1] * b[1] + a[2] * b[2]);
}

static double coord(const dmo_problem* pr, const double* c, int mesh, int axis, int v) {
  return c[((size_t)mesh * 3 + axis) * pr->P + v];
}

static void tet_vertices(const dmo_problem* pr, const double* c, int mesh, int t,
                         double X[4][3]) {
  for (int i = 0; i < 4; ++i)
    for (int a = 0; a < 3; ++a) X[i][a] = coord(pr, c, mesh, a, pr->tet[4 * t + i]);
}

/* Six times the signed volume: e1 . (e2 x e3), e_i = X_i - X_0. */
/* A tet is valid (unfolded, Sec. 2.3.4) iff 6V is positive and finite. */
static int vol_ok(double v) { return v > 0 && isfinite(v); }

static double six_vol(const double X[4][3]) {
  double e[3][3], r[3];
  for (int i = 0; i < 3; ++i)
    for (int a = 0; a < 3; ++a) e[i][a] = X[i + 1][a] - X[0][a];
  cross3(e[1], e[2], r);
  return dot3(e[0], r);
}

/* Face f (opposite local vertex f) of tet t: canonical vertices (ascending
 * point id) a,b,c; normal n = (b-a) x (c-a); inward sign s. */
typedef struct {
  double a[3], n[3];
  int s;
} dmo_face;

static void tet_faces(const dmo_problem* pr, int t, const double X[4][3], dmo_face F[4]) {
  for (int f = 0; f < 4; ++f) {
    const int8_t* fp = pr->fperm + 16 * t + 4 * f;
    const double* A = X[fp[0]];
    const double* B = X[fp[1]];
    const double* Cc = X[fp[2]];
    double u[3], w[3];
    for (int k = 0; k < 3; ++k) {
      u[k] = B[k] - A[k];
      w[k] = Cc[k] - A[k];
      F[f].a[k] = A[k];
    }
    cross3(u, w, F[f].n);
    F[f].s = fp[3];
  }
}

/* Inward-signed face value and the 3-D tie rule (Sec. 2.3.1 footnote,
 * read in 3-D): a point exactly on the face plane belongs to the side the
 * signed normal lexicographically points into, ordered (z, y, x). */
static int face_in(const dmo_face* F, const double p[3]) {
  double g = F->n[0] * (p[0] - F->a[0]) + (F->n[1] * (p[1] - F->a[1]) + F->n[2] * (p[2] - F->a[2]));
  double h = F->s > 0 ? g : -g;
  if (h > 0) return 1;
  if (h == 0) {
    double mz = F->s > 0 ? F->n[2] : -F->n[2];
    double my = F->s > 0 ? F->n[1] : -F->n[1];
    double mx = F->s > 0 ? F->n[0] : -F->n[0];
    if (mz != 0) return mz > 0;
    if (my != 0) return my > 0;
    return mx > 0;
  }
  return 0;
}

static int inside_faces(const dmo_face F[4], const double p[3]) {
  for (int f = 0; f < 4; ++f)
    if (!face_in(&F[f], p)) return 0;
  return 1;
}

/* Affine map of tet t from the "own" mesh onto the "partner" mesh,
 * displacement form:  p' = (v + d0) + G (v - own_0),
 * G = [D1 D2 D3] [r1; r2; r3] / det,  r1 = e2 x e3, r2 = e3 x e1,
 * r3 = e1 x e2, det = e1 . r1,  D_i = (par_i - par_0) - (own_i - own_0),
 * d0 = par_0 - own_0.  Equal meshes give G = 0, d0 = 0, p' = v exactly. */
typedef struct {
  double G[3][3];
  double d0[3];
  double o0[3];
  double det;
} dmo_map;

static void make_map(const double own[4][3], const double par[4][3], dmo_map* M) {
  double e[3][3], D[3][3], r[3][3];
  for (int i = 0; i < 3; ++i)
    for (int a = 0; a < 3; ++a) {
      e[i][a] = own[i + 1][a] - own[0][a];
      double f = par[i + 1][a] - par[0][a];
      D[i][a] = f - e[i][a];
    }
  cross3(e[1], e[2], r[0]);
  cross3(e[2], e[0], r[1]);
  cross3(e[0], e[1], r[2]);
  M->det = dot3(e[0], r[0]);
  double inv = 1.0 / M->det;
  for (int c = 0; c < 3; ++c)
    for (int j = 0; j < 3; ++j)
      M->G[c][j] = (D[0][c] * r[0][j] + (D[1][c] * r[1][j] + D[2][c] * r[2][j])) * inv;
  for (int a = 0; a < 3; ++a) {
    M->d0[a] = par[0][a] - own[0][a];
    M->o0[a] = own[0][a];
  }
}

static void apply_map(const dmo_map* M, const double v[3], double out[3]) {
  double q[3];
  for (int a = 0; a < 3; ++a) q[a] = v[a] - M->o0[a];
  for (int c = 0; c < 3; ++c)
    out[c] = (v[c] + M->d0[c]) + (M->G[c][0] * q[0] + (M->G[c][1] * q[1] + M->G[c][2] * q[2]));
}

/* ------------------------------------------------------- image sampling */

static double img_at(const double* img, const int n[3], int x, int y, int z) {
  return img[((size_t)z * n[1] + y) * n[0] + x];
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Trilinear sample with clamp-to-edge.  Also reports whether the sample is
 * "black": every corner that carries a nonzero weight holds 0 (Sec. 2.3.1
 * black-vs-grey rule, read on the sample's support). */
static double sample(const double* img, const int n[3], const double p[3], int* black) {
  int i0[3], i1[3];
  double f[3];
  for (int a = 0; a < 3; ++a) {
    double q = fmin(fmax(p[a], -1.0), (double)n[a]);
    double fl = floor(q);
    int i = (int)fl;
    f[a] = q - fl;
    i0[a] = clampi(i, 0, n[a] - 1);
    i1[a] = clampi(i + 1, 0, n[a] - 1);
  }
  double s = 0.0;
  int blk = 1;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
        double val = img_at(img, n, dx ? i1[0] : i0[0], dy ? i1[1] : i0[1], dz ? i1[2] : i0[2]);
        s += w * val;
        int in_support = (!dx || f[0] > 0) && (!dy || f[1] > 0) && (!dz || f[2] > 0);
        if (in_support && val != 0) blk = 0;
      }
  if (black) *black = blk;
  return s;
}

/* ------------------------------------------------------------ per-tet terms */

static int border_violations(const dmo_problem* pr, const double* c, int mesh, int v) {
  int bad = 0;
  for (int a = 0; a < 3; ++a)
    if ((pr->fixmask[v] >> a) & 1)
      if (!(coord(pr, c, mesh, a, v) == pr->rest[mesh][a * pr->P + v])) bad = 1;
  return bad;
}

static double len_mm(const double d[3], const double sp[3]) {
  double x = d[0] * sp[0], y = d[1] * sp[1], z = d[2] * sp[2];
  return sqrt(x * x + y * y + z * z);
}

/* Sec. 2.3.2: Hooke springs on 6 edges + 4 spokes, squared length change. */
static double spring_energy(const dmo_problem* pr, const double S[4][3], const double T[4][3]) {
  static const int E[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
  double e = 0.0;
  for (int k = 0; k < 6; ++k) {
    double ds[3], dt[3];
    for (int a = 0; a < 3; ++a) {
      ds[a] = S[E[k][1]][a] - S[E[k][0]][a];
      dt[a] = T[E[k][1]][a] - T[E[k][0]][a];
    }
    double d = len_mm(dt, pr->sp[1]) - len_mm(ds, pr->sp[0]);
    e += d * d;
  }
  for (int i = 0; i < 4; ++i) {
    double cs[3] = {0, 0, 0}, ct[3] = {0, 0, 0};
    for (int j = 0; j < 4; ++j)
      if (j != i)
        for (int a = 0; a < 3; ++a) {
          cs[a] += S[j][a];
          ct[a] += T[j][a];
        }
    double ds[3], dt[3];
    for (int a = 0; a < 3; ++a) {
      ds[a] = cs[a] / 3.0 - S[i][a];
      dt[a] = ct[a] / 3.0 - T[i][a];
    }
    double d = len_mm(dt, pr->sp[1]) - len_mm(ds, pr->sp[0]);
    e += d * d;
  }
  return e;
}

static int inv3(const double A[3][3], double B[3][3]) {
  double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
               A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
               A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
  if (det == 0 || !isfinite(det)) return 0;
  B[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) / det;
  B[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
  B[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
  B[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) / det;
  B[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
  B[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
  B[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) / det;
  B[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
  B[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
  return 1;
}

/* Linear-elastic model: F = D_T D_S^-1 (edge matrices in mm), taken in
 * displacement form F - I = (D_T - D_S) D_S^-1 so equal meshes give exactly
 * zero; eps = (H + H^T)/2 with H = F - I,
 * psi = mu eps:eps + lam/2 tr(eps)^2, e = V0 psi. */
static double linear_energy(const dmo_problem* pr, int t, const double S[4][3], const double T[4][3]) {
  double DS[3][3], DD[3][3], DSi[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      DS[r][c] = (S[c + 1][r] - S[0][r]) * pr->sp[0][r];
      DD[r][c] = (T[c + 1][r] - T[0][r]) * pr->sp[1][r] - DS[r][c];
    }
  if (!inv3(DS, DSi)) return 0.0;
  double H[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += DD[r][k] * DSi[k][c];
      H[r][c] = s;
    }
  double tr = 0, ee = 0;
  for (int r = 0; r < 3; ++r) {
    tr += H[r][r];
    for (int c = 0; c < 3; ++c) {
      double e = 0.5 * (H[r][c] + H[c][r]);
      ee += e * e;
    }
  }
  double psi = pr->mu * ee + 0.5 * pr->lam * tr * tr;
  return pr->rest_vol[t] * psi;
}

/* All terms of tet t for one candidate's coordinates c ([2][3][P]). */
static void tet_terms(const dmo_problem* pr, const double* c, int t, dmo_term* out) {
  double X[2][4][3];
  tet_vertices(pr, c, 0, t, X[0]);
  tet_vertices(pr, c, 1, t, X[1]);
  double vol6[2] = {six_vol(X[0]), six_vol(X[1])};
  int fold = 0;
  for (int k = 0; k < 2; ++k)
    if (!vol_ok(vol6[k])) ++fold;
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 2; ++k) fold += border_violations(pr, c, k, pr->tet[4 * t + i]);
  out->fold = fold;
  out->def = pr->model == DMO_LINEAR ? linear_energy(pr, t, X[0], X[1]) : spring_energy(pr, X[0], X[1]);
  for (int d = 0; d < 2; ++d) {
    out->ssd[d] = 0.0;
    out->cov[d] = 0;
    if (!vol_ok(vol6[d])) continue;
    const double(*own)[3] = X[d];
    const double(*par)[3] = X[1 - d];
    const int* n = pr->n[d];
    const double* Iown = pr->img[d];
    const double* Ipar = pr->img[1 - d];
    dmo_face F[4];
    tet_faces(pr, t, own, F);
    dmo_map M;
    make_map(own, par, &M);
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      lo[a] = hi[a] = own[0][a];
      for (int i = 1; i < 4; ++i) {
        lo[a] = fmin(lo[a], own[i][a]);
        hi[a] = fmax(hi[a], own[i][a]);
      }
    }
    int b0[3], b1[3];
    for (int a = 0; a < 3; ++a) {
      double l = ceil(lo[a]), h = floor(hi[a]);
      b0[a] = l < 0 ? 0 : (int)l;
      b1[a] = h > n[a] - 1 ? n[a] - 1 : (int)h;
    }
    double ssd = 0.0;
    int cov = 0;
    for (int z = b0[2]; z <= b1[2]; ++z)
      for (int y = b0[1]; y <= b1[1]; ++y)
        for (int x = b0[0]; x <= b1[0]; ++x) {
          double v[3] = {(double)x, (double)y, (double)z};
          if (!inside_faces(F, v)) continue;
          ++cov;
          double pv[3];
          apply_map(&M, v, pv);
          int blk;
          double s = sample(Ipar, pr->n[1 - d], pv, &blk);
          double o = img_at(Iown, n, x, y, z);
          double d2;
          if (pr->black_rule && ((o == 0) != blk))
            d2 = 1.0;
          else
            d2 = (o - s) * (o - s);
          ssd += d2;
        }
    out->ssd[d] = ssd;
    out->cov[d] = cov;
  }
}

/* ----------------------------------------------------------- guidance */

/* Locate p in mesh `mesh` among tets list (ascending); -1 if in none. */
static int locate(const dmo_problem* pr, const double* c, int mesh, const double p[3],
                  const int32_t* list, int nlist) {
  for (int k = 0; k < nlist; ++k) {
    int t = list ? list[k] : k;
    double X[4][3];
    tet_vertices(pr, c, mesh, t, X);
    if (!vol_ok(six_vol(X))) continue;
    dmo_face F[4];
    tet_faces(pr, t, X, F);
    if (inside_faces(F, p)) return t;
  }
  return -1;
}

/* Sec. 2.3.3: smallest squared physical distance between the mapped guidance
 * point and the points of its partner set.  mesh 0: p_i mapped
 * source->target vs the target points q_j of p_i's set (target spacing);
 * mesh 1: q_i mapped target->source vs the source points p_j (source
 * spacing).  Each pair its own set: the distance to its partner. */
static double landmark_term(const dmo_problem* pr, const double* c, int mesh, int i, int t) {
  const double* p = pr->guide + 6 * i + 3 * mesh;
  double X[2][4][3];
  tet_vertices(pr, c, mesh, t, X[0]);
  tet_vertices(pr, c, 1 - mesh, t, X[1]);
  dmo_map M;
  make_map(X[0], X[1], &M);
  double pm[3];
  apply_map(&M, p, pm);
  double best = INFINITY;
  for (int j = 0; j < pr->ng; ++j) {
    if (pr->gset ? pr->gset[j] != pr->gset[i] : j != i) continue;
    const double* q = pr->guide + 6 * j + 3 * (1 - mesh);
    double s = 0;
    for (int a = 0; a < 3; ++a) {
      double d = (pm[a] - q[a]) * pr->sp[1 - mesh][a];
      s += d * d;
    }
    if (s < best) best = s;
  }
  return best;
}

/* Guidance sets (Sec. 2.3.3): set_of[i] = set of pair i; NULL restores
 * one set per pair.  Call before evaluating. */
void dmo_set_guide_sets(void* h, const int32_t* set_of) {
  dmo_problem* pr = (dmo_problem*)h;
  free(pr->gset);
  pr->gset = NULL;
  if (set_of && pr->ng > 0) {
    pr->gset = (int32_t*)malloc(sizeof(int32_t) * pr->ng);
    memcpy(pr->gset, set_of, sizeof(int32_t) * pr->ng);
  }
}

/* ------------------------------------------------------------ problem */

static void free_trials(dmo_problem* pr) {
  free(pr->tr_cand);
  free(pr->tr_tptr);
  free(pr->tr_tets);
  free(pr->tr_terms);
  free(pr->tr_gpt_ptr);
  free(pr->tr_gpts);
  free(pr->tr_coords);
  free(pr->tr_loc);
  free(pr->tr_gterm);
  free(pr->tr_aff);
  free(pr->tr_raw);
  free(pr->tr_ntt);
  pr->tr_ntt = NULL;
  pr->tr_cand = pr->tr_tptr = pr->tr_tets = pr->tr_gpt_ptr = pr->tr_gpts = NULL;
  pr->tr_loc = pr->tr_aff = NULL;
  pr->tr_terms = NULL;
  pr->tr_coords = pr->tr_gterm = pr->tr_raw = NULL;
  pr->ntr = 0;
}

static void free_state(dmo_problem* pr) {
  free(pr->coords);
  free(pr->terms);
  free(pr->loc);
  free(pr->gterm);
  free(pr->sums);
  pr->coords = NULL;
  pr->terms = NULL;
  pr->loc = NULL;
  pr->gterm = pr->sums = NULL;
  pr->C = 0;
}

void dmo_destroy(void* h) {
  dmo_problem* pr = (dmo_problem*)h;
  if (!pr) return;
  free_trials(pr);
  free_state(pr);
  for (int k = 0; k < 2; ++k) {
    free(pr->img[k]);
    free(pr->rest[k]);
  }
  free(pr->tet);
  free(pr->fperm);
  free(pr->star_ptr);
  free(pr->star);
  free(pr->fixmask);
  free(pr->rest_vol);
  free(pr->guide);
  free(pr->gset);
  free(pr);
}

void* dmo_create(const int* nS, const int* nT, const double* spS, const double* spT,
                 const double* imgS, const double* imgT, const int* m, const double* guide,
                 int ng, int black_rule, int model, double lam, double mu) {
  dmo_problem* pr = (dmo_problem*)calloc(1, sizeof(dmo_problem));
  const int* ns[2] = {nS, nT};
  const double* sps[2] = {spS, spT};
  const double* imgs[2] = {imgS, imgT};
  for (int k = 0; k < 2; ++k) {
    for (int a = 0; a < 3; ++a) {
      pr->n[k][a] = ns[k][a];
      pr->sp[k][a] = sps[k][a];
    }
    pr->nvox[k] = (long)ns[k][0] * ns[k][1] * ns[k][2];
    pr->img[k] = (double*)malloc(sizeof(double) * pr->nvox[k]);
    memcpy(pr->img[k], imgs[k], sizeof(double) * pr->nvox[k]);
  }
  for (int a = 0; a < 3; ++a) pr->m[a] = m[a];
  pr->P = m[0] * m[1] * m[2];
  pr->ntet = dmo_num_tets(m);
  pr->tet = (int32_t*)malloc(sizeof(int32_t) * 4 * pr->ntet);
  dmo_build_tets(m, pr->tet);
  pr->fperm = (int8_t*)malloc(16 * pr->ntet);
  for (int t = 0; t < pr->ntet; ++t)
    for (int f = 0; f < 4; ++f) {
      int loc3[3], k = 0;
      for (int i = 0; i < 4; ++i)
        if (i != f) loc3[k++] = i;
      /* sort the three local indices by global point id */
      for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
          if (pr->tet[4 * t + loc3[j]] < pr->tet[4 * t + loc3[i]]) {
            int tmp = loc3[i];
            loc3[i] = loc3[j];
            loc3[j] = tmp;
          }
      int perm[4] = {loc3[0], loc3[1], loc3[2], f};
      int8_t* fp = pr->fperm + 16 * t + 4 * f;
      fp[0] = (int8_t)loc3[0];
      fp[1] = (int8_t)loc3[1];
      fp[2] = (int8_t)loc3[2];
      fp[3] = (int8_t)perm_parity(perm);
    }
  /* point -> tets, ascending (Sec. 2.2 dependency structure) */
  pr->star_ptr = (int32_t*)calloc(pr->P + 1, sizeof(int32_t));
  for (int t = 0; t < pr->ntet; ++t)
    for (int i = 0; i < 4; ++i) pr->star_ptr[pr->tet[4 * t + i] + 1]++;
  for (int v = 0; v < pr->P; ++v) pr->star_ptr[v + 1] += pr->star_ptr[v];
  pr->star = (int32_t*)malloc(sizeof(int32_t) * 4 * pr->ntet);
  int32_t* fill = (int32_t*)malloc(sizeof(int32_t) * pr->P);
  memcpy(fill, pr->star_ptr, sizeof(int32_t) * pr->P);
  for (int t = 0; t < pr->ntet; ++t)
    for (int i = 0; i < 4; ++i) pr->star[fill[pr->tet[4 * t + i]]++] = t;
  free(fill);
  /* rest lattice: point (a,b,c) at -0.5 + a*n/(m-1); border axes fixed */
  pr->fixmask = (uint8_t*)calloc(pr->P, 1);
  for (int k = 0; k < 2; ++k) pr->rest[k] = (double*)malloc(sizeof(double) * 3 * pr->P);
  for (int c = 0; c < m[2]; ++c)
    for (int b = 0; b < m[1]; ++b)
      for (int a = 0; a < m[0]; ++a) {
        int v = point_id(m, a, b, c);
        int idx[3] = {a, b, c};
        for (int ax = 0; ax < 3; ++ax) {
          if (idx[ax] == 0 || idx[ax] == m[ax] - 1) pr->fixmask[v] |= (uint8_t)(1 << ax);
          for (int k = 0; k < 2; ++k)
            pr->rest[k][ax * pr->P + v] = (double)idx[ax] * (double)pr->n[k][ax] / (double)(m[ax] - 1) - 0.5;
        }
      }
  pr->rest_vol = (double*)malloc(sizeof(double) * pr->ntet);
  pr->rest_vol_sum = 0;
  for (int t = 0; t < pr->ntet; ++t) {
    double X[4][3];
    for (int i = 0; i < 4; ++i)
      for (int a = 0; a < 3; ++a) X[i][a] = pr->rest[0][a * pr->P + pr->tet[4 * t + i]] * pr->sp[0][a];
    pr->rest_vol[t] = fabs(six_vol(X)) / 6.0;
    pr->rest_vol_sum += pr->rest_vol[t];
  }
  pr->black_rule = black_rule;
  pr->model = model;
  pr->lam = lam;
  pr->mu = mu;
  pr->ng = ng;
  pr->guide = (double*)malloc(sizeof(double) * 6 * (ng > 0 ? ng : 1));
  if (ng > 0) memcpy(pr->guide, guide, sizeof(double) * 6 * ng);
  return pr;
}

int dmo_ntet(void* h) { return ((dmo_problem*)h)->ntet; }
int dmo_npoints(void* h) { return ((dmo_problem*)h)->P; }
void dmo_get_tets(void* h, int32_t* out) {
  dmo_problem* pr = (dmo_problem*)h;
  memcpy(out, pr->tet, sizeof(int32_t) * 4 * pr->ntet);
}
void dmo_get_star(void* h, int32_t* ptr, int32_t* idx) {
  dmo_problem* pr = (dmo_problem*)h;
  memcpy(ptr, pr->star_ptr, sizeof(int32_t) * (pr->P + 1));
  memcpy(idx, pr->star, sizeof(int32_t) * 4 * pr->ntet);
}
void dmo_get_face_perm(void* h, int8_t* out) {
  dmo_problem* pr = (dmo_problem*)h;
  memcpy(out, pr->fperm, 16 * pr->ntet);
}
void dmo_rest_coords(void* h, int mesh, double* out) {
  dmo_problem* pr = (dmo_problem*)h;
  memcpy(out, pr->rest[mesh], sizeof(double) * 3 * pr->P);
}

static double def_norm(const dmo_problem* pr) {
  return pr->model == DMO_LINEAR ? pr->rest_vol_sum : 10.0 * pr->ntet;
}

static void normalise(const dmo_problem* pr, const double raw[4], double out[4]) {
  out[0] = raw[0] / (double)(pr->nvox[0] + pr->nvox[1]);
  out[1] = raw[1] / def_norm(pr);
  out[2] = pr->ng > 0 ? raw[2] / (2.0 * pr->ng) : 0.0;
  out[3] = raw[3];
}

/* Full evaluation of C candidates; (re)initialises the population state. */
int dmo_eval_full(void* h, int C, const double* coords, double* obj) {
  dmo_problem* pr = (dmo_problem*)h;
  free_trials(pr);
  free_state(pr);
  pr->C = C;
  size_t csz = (size_t)6 * pr->P;
  pr->coords = (double*)malloc(sizeof(double) * csz * C);
  memcpy(pr->coords, coords, sizeof(double) * csz * C);
  pr->terms = (dmo_term*)malloc(sizeof(dmo_term) * (size_t)C * pr->ntet);
  int ngs = pr->ng > 0 ? pr->ng : 1;
  pr->loc = (int32_t*)malloc(sizeof(int32_t) * (size_t)C * 2 * ngs);
  pr->gterm = (double*)malloc(sizeof(double) * (size_t)C * 2 * ngs);
  pr->sums = (double*)malloc(sizeof(double) * 4 * C);
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 1)
  for (int ci = 0; ci < C; ++ci) {
    const double* c = pr->coords + csz * ci;
    dmo_term* T = pr->terms + (size_t)ci * pr->ntet;
    double raw[4] = {0, 0, 0, 0};
    for (int t = 0; t < pr->ntet; ++t) {
      tet_terms(pr, c, t, &T[t]);
      raw[0] += T[t].ssd[0] + T[t].ssd[1];
      raw[1] += T[t].def;
      raw[3] += T[t].fold;
    }
    for (int k = 0; k < 2; ++k)
      for (int i = 0; i < pr->ng; ++i) {
        const double* p = pr->guide + 6 * i + 3 * k;
        int t = locate(pr, c, k, p, NULL, pr->ntet);
        size_t li = ((size_t)ci * 2 + k) * ngs + i;
        pr->loc[li] = t;
        pr->gterm[li] = t >= 0 ? landmark_term(pr, c, k, i, t) : 0.0;
        if (t < 0) raw[3] += 1;
        raw[2] += pr->gterm[li];
      }
    memcpy(pr->sums + 4 * ci, raw, sizeof(raw));
    normalise(pr, raw, obj + 4 * ci);
  }
  return 0;
}

static int in_sorted(const int32_t* a, int n, int v) {
  int lo = 0, hi = n - 1;
  while (lo <= hi) {
    int mid = (lo + hi) / 2;
    if (a[mid] == v) return 1;
    if (a[mid] < v) lo = mid + 1;
    else hi = mid - 1;
  }
  return 0;
}

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* Touched tets of a point group: sorted union of the points' stars. */
static int touched_tets(const dmo_problem* pr, const int32_t* pts, int np, int32_t* out) {
  int n = 0;
  for (int k = 0; k < np; ++k)
    for (int j = pr->star_ptr[pts[k]]; j < pr->star_ptr[pts[k] + 1]; ++j) out[n++] = pr->star[j];
  qsort(out, n, sizeof(int32_t), cmp_i32);
  int u = 0;
  for (int k = 0; k < n; ++k)
    if (u == 0 || out[u - 1] != out[k]) out[u++] = out[k];
  return u;
}

/* Partial evaluation (Sec. 2.2): trial k moves the points gpts[gptr[k]..]
 * of candidate cand[k] to tcoords (per trial [2][3][npts]); only touched
 * tets and the landmarks located in them are re-evaluated.  The state is
 * not changed; dmo_commit applies accepted trials. */
int dmo_eval_partial(void* h, int ntr, const int32_t* cand, const int32_t* gptr,
                     const int32_t* gpts, const double* tcoords, double* obj) {
  dmo_problem* pr = (dmo_problem*)h;
  free_trials(pr);
  for (int k = 0; k < ntr; ++k)
    if (cand[k] < 0 || cand[k] >= pr->C) return -1;
  int ngs = pr->ng > 0 ? pr->ng : 1;
  pr->ntr = ntr;
  int totpts = gptr[ntr];
  pr->tr_cand = (int32_t*)malloc(sizeof(int32_t) * (ntr > 0 ? ntr : 1));
  memcpy(pr->tr_cand, cand, sizeof(int32_t) * ntr);
  pr->tr_gpt_ptr = (int32_t*)malloc(sizeof(int32_t) * (ntr + 1));
  memcpy(pr->tr_gpt_ptr, gptr, sizeof(int32_t) * (ntr + 1));
  pr->tr_gpts = (int32_t*)malloc(sizeof(int32_t) * (totpts > 0 ? totpts : 1));
  memcpy(pr->tr_gpts, gpts, sizeof(int32_t) * totpts);
  pr->tr_coords = (double*)malloc(sizeof(double) * 6 * (totpts > 0 ? totpts : 1));
  memcpy(pr->tr_coords, tcoords, sizeof(double) * 6 * totpts);
  pr->tr_tptr = (int32_t*)malloc(sizeof(int32_t) * (ntr + 1));
  pr->tr_tptr[0] = 0;
  for (int k = 0; k < ntr; ++k) {
    int s = 0;
    for (int j = gptr[k]; j < gptr[k + 1]; ++j) s += pr->star_ptr[gpts[j] + 1] - pr->star_ptr[gpts[j]];
    pr->tr_tptr[k + 1] = pr->tr_tptr[k] + s; /* upper bound, compacted below */
  }
  pr->tr_tets = (int32_t*)malloc(sizeof(int32_t) * (pr->tr_tptr[ntr] > 0 ? pr->tr_tptr[ntr] : 1));
  pr->tr_terms = (dmo_term*)malloc(sizeof(dmo_term) * (pr->tr_tptr[ntr] > 0 ? pr->tr_tptr[ntr] : 1));
  pr->tr_loc = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ntr > 0 ? ntr : 1) * 2 * ngs);
  pr->tr_gterm = (double*)malloc(sizeof(double) * (size_t)(ntr > 0 ? ntr : 1) * 2 * ngs);
  pr->tr_aff = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ntr > 0 ? ntr : 1) * 2 * ngs);
  pr->tr_raw = (double*)malloc(sizeof(double) * 4 * (ntr > 0 ? ntr : 1));
  int32_t* ntt = (int32_t*)malloc(sizeof(int32_t) * (ntr > 0 ? ntr : 1));
  size_t csz = (size_t)6 * pr->P;
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 1)
  for (int k = 0; k < ntr; ++k) {
    int ci = cand[k];
    double* c = (double*)malloc(sizeof(double) * csz);
    memcpy(c, pr->coords + csz * ci, sizeof(double) * csz);
    int np = gptr[k + 1] - gptr[k];
    const int32_t* pts = gpts + gptr[k];
    const double* tc = tcoords + 6 * (size_t)gptr[k];
    for (int mesh = 0; mesh < 2; ++mesh)
      for (int a = 0; a < 3; ++a)
        for (int j = 0; j < np; ++j) c[(mesh * 3 + a) * pr->P + pts[j]] = tc[(mesh * 3 + a) * np + j];
    int32_t* tl = pr->tr_tets + pr->tr_tptr[k];
    int nt = touched_tets(pr, pts, np, tl);
    ntt[k] = nt;
    dmo_term* TT = pr->tr_terms + pr->tr_tptr[k];
    const dmo_term* old = pr->terms + (size_t)ci * pr->ntet;
    double raw[4];
    memcpy(raw, pr->sums + 4 * ci, sizeof(raw));
    for (int j = 0; j < nt; ++j) {
      const dmo_term* o = &old[tl[j]];
      raw[0] -= o->ssd[0] + o->ssd[1];
      raw[1] -= o->def;
      raw[3] -= o->fold;
    }
    for (int j = 0; j < nt; ++j) {
      tet_terms(pr, c, tl[j], &TT[j]);
      raw[0] += TT[j].ssd[0] + TT[j].ssd[1];
      raw[1] += TT[j].def;
      raw[3] += TT[j].fold;
    }
    for (int mesh = 0; mesh < 2; ++mesh)
      for (int i = 0; i < pr->ng; ++i) {
        size_t li = ((size_t)ci * 2 + mesh) * ngs + i;
        size_t ti = ((size_t)k * 2 + mesh) * ngs + i;
        int t_old = pr->loc[li];
        int aff = t_old < 0 || in_sorted(tl, nt, t_old);
        pr->tr_aff[ti] = aff;
        pr->tr_loc[ti] = t_old;
        pr->tr_gterm[ti] = pr->gterm[li];
        if (!aff) continue;
        const double* p = pr->guide + 6 * i + 3 * mesh;
        int t = locate(pr, c, mesh, p, tl, nt);
        double gt = t >= 0 ? landmark_term(pr, c, mesh, i, t) : 0.0;
        raw[2] += gt - pr->gterm[li];
        raw[3] += (t < 0 ? 1 : 0) - (t_old < 0 ? 1 : 0);
        pr->tr_loc[ti] = t;
        pr->tr_gterm[ti] = gt;
      }
    memcpy(pr->tr_raw + 4 * k, raw, sizeof(raw));
    normalise(pr, raw, obj + 4 * k);
    free(c);
  }
  pr->tr_ntt = ntt;
  return 0;
}

/* Apply the accepted trials of the last partial evaluation.  Accepted trials
 * of one candidate must touch disjoint tet sets (their changes are then
 * independent, Sec. 2.2); otherwise nothing is applied and -1 is returned. */
int dmo_commit(void* h, const uint8_t* accept) {
  dmo_problem* pr = (dmo_problem*)h;
  int ngs = pr->ng > 0 ? pr->ng : 1;
  for (int k = 0; k < pr->ntr; ++k) {
    if (!accept[k]) continue;
    for (int j = k + 1; j < pr->ntr; ++j) {
      if (!accept[j] || pr->tr_cand[j] != pr->tr_cand[k]) continue;
      const int32_t* a = pr->tr_tets + pr->tr_tptr[k];
      const int32_t* b = pr->tr_tets + pr->tr_tptr[j];
      for (int x = 0; x < pr->tr_ntt[k]; ++x)
        if (in_sorted(b, pr->tr_ntt[j], a[x])) return -1;
    }
  }
  size_t csz = (size_t)6 * pr->P;
  for (int k = 0; k < pr->ntr; ++k) {
    if (!accept[k]) continue;
    int ci = pr->tr_cand[k];
    double* c = pr->coords + csz * ci;
    int np = pr->tr_gpt_ptr[k + 1] - pr->tr_gpt_ptr[k];
    const int32_t* pts = pr->tr_gpts + pr->tr_gpt_ptr[k];
    const double* tc = pr->tr_coords + 6 * (size_t)pr->tr_gpt_ptr[k];
    for (int mesh = 0; mesh < 2; ++mesh)
      for (int a = 0; a < 3; ++a)
        for (int j = 0; j < np; ++j) c[(mesh * 3 + a) * pr->P + pts[j]] = tc[(mesh * 3 + a) * np + j];
    double* s = pr->sums + 4 * ci;
    /* the trial's raw sums were formed from the pre-wave sums; with disjoint
     * accepted trials the change of each one adds independently */
    dmo_term* T = pr->terms + (size_t)ci * pr->ntet;
    const int32_t* tl = pr->tr_tets + pr->tr_tptr[k];
    const dmo_term* TT = pr->tr_terms + pr->tr_tptr[k];
    double delta[4] = {0, 0, 0, 0};
    for (int j = 0; j < pr->tr_ntt[k]; ++j) {
      const dmo_term* o = &T[tl[j]];
      delta[0] += (TT[j].ssd[0] + TT[j].ssd[1]) - (o->ssd[0] + o->ssd[1]);
      delta[1] += TT[j].def - o->def;
      delta[3] += TT[j].fold - o->fold;
      T[tl[j]] = TT[j];
    }
    for (int mesh = 0; mesh < 2; ++mesh)
      for (int i = 0; i < pr->ng; ++i) {
        size_t ti = ((size_t)k * 2 + mesh) * ngs + i;
        size_t li = ((size_t)ci * 2 + mesh) * ngs + i;
        if (!pr->tr_aff[ti]) continue;
        delta[2] += pr->tr_gterm[ti] - pr->gterm[li];
        delta[3] += (pr->tr_loc[ti] < 0 ? 1 : 0) - (pr->loc[li] < 0 ? 1 : 0);
        pr->loc[li] = pr->tr_loc[ti];
        pr->gterm[li] = pr->tr_gterm[ti];
      }
    for (int q = 0; q < 4; ++q) s[q] += delta[q];
  }
  return 0;
}

void dmo_get_objectives(void* h, int n, const int32_t* cands, double* out) {
  dmo_problem* pr = (dmo_problem*)h;
  for (int k = 0; k < n; ++k) normalise(pr, pr->sums + 4 * cands[k], out + 4 * k);
}

void dmo_get_raw(void* h, int c, double* out) { memcpy(out, ((dmo_problem*)h)->sums + 4 * c, 4 * sizeof(double)); }

void dmo_get_coords(void* h, int c, double* out) {
  dmo_problem* pr = (dmo_problem*)h;
  memcpy(out, pr->coords + (size_t)6 * pr->P * c, sizeof(double) * 6 * pr->P);
}

void dmo_get_terms(void* h, int c, double* ssd, int32_t* cov, double* def, int32_t* fold) {
  dmo_problem* pr = (dmo_problem*)h;
  const dmo_term* T = pr->terms + (size_t)c * pr->ntet;
  for (int t = 0; t < pr->ntet; ++t) {
    ssd[2 * t] = T[t].ssd[0];
    ssd[2 * t + 1] = T[t].ssd[1];
    cov[2 * t] = T[t].cov[0];
    cov[2 * t + 1] = T[t].cov[1];
    def[t] = T[t].def;
    fold[t] = T[t].fold;
  }
}

void dmo_get_landmarks(void* h, int c, int32_t* loc, double* gterm) {
  dmo_problem* pr = (dmo_problem*)h;
  int ngs = pr->ng > 0 ? pr->ng : 1;
  for (int mesh = 0; mesh < 2; ++mesh)
    for (int i = 0; i < pr->ng; ++i) {
      loc[mesh * pr->ng + i] = pr->loc[((size_t)c * 2 + mesh) * ngs + i];
      gterm[mesh * pr->ng + i] = pr->gterm[((size_t)c * 2 + mesh) * ngs + i];
    }
}

/* Trial outputs of the last partial evaluation: touched tets and their new
 * terms for trial k. Returns the touched-set size. */
int dmo_get_trial(void* h, int k, int32_t* tets, double* ssd, int32_t* cov, double* def, int32_t* fold) {
  dmo_problem* pr = (dmo_problem*)h;
  int nt = pr->tr_ntt[k];
  const int32_t* tl = pr->tr_tets + pr->tr_tptr[k];
  const dmo_term* TT = pr->tr_terms + pr->tr_tptr[k];
  for (int j = 0; j < nt; ++j) {
    if (tets) tets[j] = tl[j];
    if (ssd) {
      ssd[2 * j] = TT[j].ssd[0];
      ssd[2 * j + 1] = TT[j].ssd[1];
    }
    if (cov) {
      cov[2 * j] = TT[j].cov[0];
      cov[2 * j + 1] = TT[j].cov[1];
    }
    if (def) def[j] = TT[j].def;
    if (fold) fold[j] = TT[j].fold;
  }
  return nt;
}

/* ---------------------------------------------- single-item entry points */

/* coords: one candidate [2][3][P]. */
void dmo_tet_terms(void* h, const double* coords, int t, double* ssd2, int32_t* cov2, double* def,
                   int32_t* fold) {
  dmo_term T;
  tet_terms((dmo_problem*)h, coords, t, &T);
  ssd2[0] = T.ssd[0];
  ssd2[1] = T.ssd[1];
  cov2[0] = T.cov[0];
  cov2[1] = T.cov[1];
  *def = T.def;
  *fold = T.fold;
}

int dmo_inside(void* h, int mesh, const double* coords, int t, const double* p) {
  dmo_problem* pr = (dmo_problem*)h;
  double X[4][3];
  tet_vertices(pr, coords, mesh, t, X);
  if (!vol_ok(six_vol(X))) return 0;
  dmo_face F[4];
  tet_faces(pr, t, X, F);
  return inside_faces(F, p);
}

/* Voxel coverage of tet t in mesh `mesh`, one flag per voxel of the own
 * image (brute force over every voxel, not only the bounding box). */
void dmo_coverage_mask(void* h, int mesh, const double* coords, int t, uint8_t* mask) {
  dmo_problem* pr = (dmo_problem*)h;
  const int* n = pr->n[mesh];
  double X[4][3];
  tet_vertices(pr, coords, mesh, t, X);
  int ok = vol_ok(six_vol(X));
  dmo_face F[4];
  tet_faces(pr, t, X, F);
  for (int z = 0; z < n[2]; ++z)
    for (int y = 0; y < n[1]; ++y)
      for (int x = 0; x < n[0]; ++x) {
        double v[3] = {(double)x, (double)y, (double)z};
        mask[((size_t)z * n[1] + y) * n[0] + x] = (uint8_t)(ok && inside_faces(F, v));
      }
}

void dmo_map_point(void* h, int dir, const double* coords, int t, const double* v, double* out) {
  dmo_problem* pr = (dmo_problem*)h;
  double X[2][4][3];
  tet_vertices(pr, coords, dir, t, X[0]);
  tet_vertices(pr, coords, 1 - dir, t, X[1]);
  dmo_map M;
  make_map(X[0], X[1], &M);
  apply_map(&M, v, out);
}

double dmo_sample(void* h, int img, const double* p, int32_t* black) {
  dmo_problem* pr = (dmo_problem*)h;
  int b;
  double s = sample(pr->img[img], pr->n[img], p, &b);
  if (black) *black = b;
  return s;
}

double dmo_six_vol(void* h, int mesh, const double* coords, int t) {
  dmo_problem* pr = (dmo_problem*)h;
  double X[4][3];
  tet_vertices(pr, coords, mesh, t, X);
  return six_vol(X);
}

/* ------------------------------------------------------------------ refinement
 * Grid multi-resolution (Sec. 2.4): every cube cell of both meshes gains a
 * point in the middle of each edge, in the middle of each face and at its
 * centre, so m points per axis become 2m - 1.  Fine point (A, B, C) sits on
 * coarse point (A/2, B/2, C/2) when all its indices are even; otherwise it is
 * the mean of the coarse points at the corners of the edge, face or cube it
 * lies in (a deformed face is non-planar: the mean of its 4 corners; the
 * cube's centre of mass: the mean of its 8 corners).  Summation order, which
 * the GPU follows as well: recursive halves along the odd axes taken in the
 * order z, y, x, i.e. ((c_000 + c_001) + (c_010 + c_011)) + (...), then one
 * exact scaling by 2^-k for k odd axes.
 * coarse: [ncand][2][3][mx*my*mz]; fine: [ncand][2][3][Mx*My*Mz]. */
static double refine_sum(const double* v, const int* m, int A, int B, int Cz, int level) {
  /* level 0: z, 1: y, 2: x; recurse on odd fine indices */
  const int idx[3] = {A, B, Cz};
  if (level == 3) return v[(A / 2) + m[0] * ((B / 2) + m[1] * (Cz / 2))];
  int ax = 2 - level; /* z first, then y, then x */
  if (idx[ax] & 1) {
    int lo[3] = {A, B, Cz}, hi[3] = {A, B, Cz};
    lo[ax] -= 1;
    hi[ax] += 1;
    return refine_sum(v, m, lo[0], lo[1], lo[2], level + 1) + refine_sum(v, m, hi[0], hi[1], hi[2], level + 1);
  }
  return refine_sum(v, m, A, B, Cz, level + 1);
}

int dmo_refine(const double* coarse, int ncand, int mx, int my, int mz, double* fine) {
  if (ncand < 0 || mx < 2 || my < 2 || mz < 2) return -1;
  const int m[3] = {mx, my, mz};
  const int M[3] = {2 * mx - 1, 2 * my - 1, 2 * mz - 1};
  const long P = (long)mx * my * mz, PF = (long)M[0] * M[1] * M[2];
  for (long cma = 0; cma < (long)ncand * 6; ++cma) {
    const double* v = coarse + cma * P;
    double* out = fine + cma * PF;
    for (int Cz = 0; Cz < M[2]; ++Cz)
      for (int B = 0; B < M[1]; ++B)
        for (int A = 0; A < M[0]; ++A) {
          int k = (A & 1) + (B & 1) + (Cz & 1);
          double s = refine_sum(v, m, A, B, Cz, 0);
          out[A + (long)M[0] * (B + (long)M[1] * Cz)] = s * (k == 0 ? 1.0 : k == 1 ? 0.5 : k == 2 ? 0.25 : 0.125);
        }
  }
  return 0;
}

/* ------------------------------------------------------------------ link test
 * The paper's folding check (Sec. 2.3.4): a point violates the constraint if
 * it lies outside the polyhedron formed by the faces of its star's tets that
 * do not contain it (its link).  Inside / outside by the parity of the
 * crossings of a ray from the point.  Border points (one fixed axis) move in
 * their border plane and are tested in 2-D against the polygon of the star
 * triangles' edges that lie in that plane; points on a border edge (two fixed
 * axes) must lie strictly between their two lattice neighbours along the free
 * axis; corners are fixed.
 * Ray directions: (1, RAY_Y, RAY_Z) in 3-D and (1, RAY_Y) over the two free
 * axes (in axis order) in 2-D, fixed "generic" constants so that a ray meets a
 * triangle edge or a segment end only on a set of measure zero.  Triangle
 * crossing (Moeller & Trumbore, "Fast, minimum storage ray-triangle
 * intersection", 1997): closed triangle, strictly ahead of the origin.
 * Segment crossing: segment parameter in [0, 1), strictly ahead.  FP64, one
 * rounding per operation in the order written. */
#define RAY_Y 0.7548776662466927
#define RAY_Z 0.5698402909980532

static int ray_hits_triangle(const double* o, const double* a, const double* b, const double* c) {
  const double R[3] = {1.0, RAY_Y, RAY_Z};
  double e1[3], e2[3], tv[3], pv[3], qv[3];
  for (int k = 0; k < 3; ++k) {
    e1[k] = b[k] - a[k];
    e2[k] = c[k] - a[k];
    tv[k] = o[k] - a[k];
  }
  pv[0] = R[1] * e2[2] - R[2] * e2[1];
  pv[1] = R[2] * e2[0] - R[0] * e2[2];
  pv[2] = R[0] * e2[1] - R[1] * e2[0];
  const double det = (e1[0] * pv[0] + e1[1] * pv[1]) + e1[2] * pv[2];
  if (det == 0.0) return 0;
  const double inv = 1.0 / det;
  const double u = ((tv[0] * pv[0] + tv[1] * pv[1]) + tv[2] * pv[2]) * inv;
  if (u < 0.0 || u > 1.0) return 0;
  qv[0] = tv[1] * e1[2] - tv[2] * e1[1];
  qv[1] = tv[2] * e1[0] - tv[0] * e1[2];
  qv[2] = tv[0] * e1[1] - tv[1] * e1[0];
  const double w = ((R[0] * qv[0] + R[1] * qv[1]) + R[2] * qv[2]) * inv;
  if (w < 0.0 || u + w > 1.0) return 0;
  const double t = ((e2[0] * qv[0] + e2[1] * qv[1]) + e2[2] * qv[2]) * inv;
  return t > 0.0;
}

/* 2-D: ray o + s (1, RAY_Y), s > 0, against segment p + r (q - p), 0 <= r < 1 */
static int ray_hits_segment(const double* o, const double* p, const double* q) {
  const double dx = q[0] - p[0], dy = q[1] - p[1];
  const double den = 1.0 * dy - RAY_Y * dx;
  if (den == 0.0) return 0;
  const double px = p[0] - o[0], py = p[1] - o[1];
  const double s = (px * dy - py * dx) / den;
  const double r = (px * RAY_Y - py * 1.0) / den;
  return s > 0.0 && r >= 0.0 && r < 1.0;
}

static int lattice_index(const int* m, int v, int ax) {
  return ax == 0 ? v % m[0] : ax == 1 ? (v / m[0]) % m[1] : v / (m[0] * m[1]);
}

/* 1 if point v of mesh `mesh` (coords c = [2][3][P]) violates its link */
static int link_violation(const dmo_problem* pr, const double* c, int mesh, int v) {
  const int P = pr->P;
  const double* X = c + (size_t)mesh * 3 * P;
  const uint8_t fm = pr->fixmask[v];
  const int nfix = (fm & 1) + ((fm >> 1) & 1) + ((fm >> 2) & 1);
  double o[3] = {X[v], X[P + v], X[2 * P + v]};
  if (nfix == 3) return 0;
  if (nfix == 2) {
    const int ax = !(fm & 1) ? 0 : !(fm & 2) ? 1 : 2;
    const int step = ax == 0 ? 1 : ax == 1 ? pr->m[0] : pr->m[0] * pr->m[1];
    const double lo = X[(size_t)ax * P + v - step], hi = X[(size_t)ax * P + v + step];
    return !(lo < o[ax] && o[ax] < hi);
  }
  int hits = 0;
  if (nfix == 0) {
    for (int s = pr->star_ptr[v]; s < pr->star_ptr[v + 1]; ++s) {
      const int t = pr->star[s];
      double V[3][3];
      int n = 0;
      for (int i = 0; i < 4; ++i) {
        const int w = pr->tet[4 * t + i];
        if (w == v) continue;
        for (int a = 0; a < 3; ++a) V[n][a] = X[(size_t)a * P + w];
        ++n;
      }
      hits += ray_hits_triangle(o, V[0], V[1], V[2]);
    }
    return !(hits & 1);
  }
  /* one fixed axis f: the star triangles lying in v's border plane */
  const int f = (fm & 1) ? 0 : (fm & 2) ? 1 : 2;
  const int a1 = f == 0 ? 1 : 0, a2 = f == 2 ? 1 : 2;
  const int fv = lattice_index(pr->m, v, f);
  const double o2[2] = {o[a1], o[a2]};
  for (int s = pr->star_ptr[v]; s < pr->star_ptr[v + 1]; ++s) {
    const int t = pr->star[s];
    int ids[2], n = 0, ok = 1;
    for (int i = 0; i < 4; ++i) {
      const int w = pr->tet[4 * t + i];
      if (w == v) continue;
      if (lattice_index(pr->m, w, f) == fv) {
        if (n < 2) ids[n] = w;
        ++n;
      }
    }
    if (n != 2) ok = 0;
    if (!ok) continue;
    const double p[2] = {X[(size_t)a1 * P + ids[0]], X[(size_t)a2 * P + ids[0]]};
    const double q[2] = {X[(size_t)a1 * P + ids[1]], X[(size_t)a2 * P + ids[1]]};
    hits += ray_hits_segment(o2, p, q);
  }
  return !(hits & 1);
}

/* 1 if point v of `mesh` lies outside its link */
int dmo_link_point(void* h, const double* coords, int mesh, int v) {
  return link_violation((const dmo_problem*)h, coords, mesh, v);
}

/* out2[mesh] = number of points of that mesh outside their link */
void dmo_link_violations(void* h, const double* coords, int32_t* out2) {
  const dmo_problem* pr = (const dmo_problem*)h;
  for (int mesh = 0; mesh < 2; ++mesh) {
    int n = 0;
    for (int v = 0; v < pr->P; ++v) n += link_violation(pr, coords, mesh, v);
    out2[mesh] = n;
  }
}
