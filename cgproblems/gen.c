/*
 * Seeded synthetic SPD test problems in CSR form (int32 indices, fp64 values).
 *
 * This module is the one piece of code that both the CG oracle and the CUDA
 * path consume: it builds the inputs A and x* and nothing else.  It holds no
 * arithmetic of the conjugate-gradient method (no SpMV, no dot products, no
 * vector updates); right-hand sides b = A x* are formed by whichever side
 * uses the matrix.
 *
 * The paper measures on SuiteSparse matrices (Sec. 4.1); those are not
 * reproduced here.  Every matrix below is symmetric positive definite by
 * construction with Dirichlet boundaries: a neighbour outside the domain is
 * dropped from the row but its coupling weight stays on the diagonal.
 * Within each row the column indices are strictly increasing and the
 * diagonal is always stored.
 *
 * Random numbers come from a counter-based SplitMix64 (Steele, Lea and
 * Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
 * value(seed, c) = mix64(seed + (c + 1) * 0x9E3779B97F4A7C15).  Normal
 * deviates use the Box-Muller transform on two consecutive counters.
 *
 * Every builder has a *_size() call that reports n and nnz and a *_fill()
 * call that writes caller-allocated arrays rowptr[n+1], colind[nnz],
 * vals[nnz].  All return 0 on success and a negative value on bad arguments.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t gen_splitmix64(uint64_t seed, uint64_t ctr) {
  return mix64(seed + (ctr + 1) * GOLDEN);
}

/* uniform in [0, 1) with 53 random bits */
static double u01(uint64_t seed, uint64_t ctr) {
  return (double)(gen_splitmix64(seed, ctr) >> 11) * 0x1.0p-53;
}

/* uniform in (0, 1] */
static double u01_open0(uint64_t seed, uint64_t ctr) {
  return (double)((gen_splitmix64(seed, ctr) >> 11) + 1) * 0x1.0p-53;
}

/* standard normal deviate number `ctr` of the stream (Box-Muller, cosine branch) */
double gen_normal(uint64_t seed, uint64_t ctr) {
  const double two_pi = 6.283185307179586476925286766559;
  double u1 = u01_open0(seed, 2 * ctr);
  double u2 = u01(seed, 2 * ctr + 1);
  return sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
}

/* x*_i uniform in [-1, 1) */
int gen_uniform_pm1(int64_t n, uint64_t seed, double* out) {
  if (n < 0 || (n > 0 && !out)) return -1;
  for (int64_t i = 0; i < n; ++i) out[i] = 2.0 * u01(seed, (uint64_t)i) - 1.0;
  return 0;
}

/* ------------------------------------------------------------------ */
/* 2-D grids: 5-point and 9-point anisotropic graph Laplacians         */
/* ------------------------------------------------------------------ */
/* Unknown (x, y), 0 <= x, y < N, row index y*N + x.  5-point couplings:
 * eps along x, 1 along y.  9-point adds the four diagonal couplings with
 * weight (1 + eps)/4.  Diagonal = sum of all coupling weights, including
 * those to outside (Dirichlet) neighbours: 2eps + 2 (5-point) and
 * 3eps + 3 (9-point).  eps = 1, 5-point gives the textbook (4, -1) stencil. */

static int lap2d_check(int64_t N, int points, double eps) {
  if (N < 1 || N > 46340) return -1;
  if (points != 5 && points != 9) return -1;
  if (!(eps > 0.0)) return -1;
  return 0;
}

int gen_lap2d_size(int64_t N, int points, double eps, int64_t* n, int64_t* nnz) {
  if (lap2d_check(N, points, eps)) return -1;
  int64_t cnt = 0;
  for (int64_t y = 0; y < N; ++y)
    for (int64_t x = 0; x < N; ++x)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          if (points == 5 && dx != 0 && dy != 0) continue;
          int64_t xx = x + dx, yy = y + dy;
          if (xx < 0 || xx >= N || yy < 0 || yy >= N) continue;
          ++cnt;
        }
  *n = N * N;
  *nnz = cnt;
  return 0;
}

int gen_lap2d_fill(int64_t N, int points, double eps,
                   int32_t* rowptr, int32_t* colind, double* vals) {
  if (lap2d_check(N, points, eps)) return -1;
  const double wd = (1.0 + eps) / 4.0;
  const double diag = (points == 5) ? (2.0 * eps + 2.0) : (3.0 * eps + 3.0);
  int64_t k = 0;
  rowptr[0] = 0;
  for (int64_t y = 0; y < N; ++y)
    for (int64_t x = 0; x < N; ++x) {
      /* (dy, dx) in row-major order visits columns in increasing order */
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          if (points == 5 && dx != 0 && dy != 0) continue;
          int64_t xx = x + dx, yy = y + dy;
          if (xx < 0 || xx >= N || yy < 0 || yy >= N) continue;
          double v;
          if (dx == 0 && dy == 0) v = diag;
          else if (dy == 0) v = -eps;
          else if (dx == 0) v = -1.0;
          else v = -wd;
          colind[k] = (int32_t)(yy * N + xx);
          vals[k] = v;
          ++k;
        }
      rowptr[y * N + x + 1] = (int32_t)k;
    }
  return 0;
}

/* ------------------------------------------------------------------ */
/* 3-D 7-point unit Laplacian (diagonal 6, couplings -1)               */
/* ------------------------------------------------------------------ */
/* Unknown (x, y, z), row index (z*N + y)*N + x. */

int gen_lap3d7_size(int64_t N, int64_t* n, int64_t* nnz) {
  if (N < 1 || N > 1290) return -1;
  int64_t n_ = N * N * N;
  /* 7 per node minus one per missing face neighbour: 6 faces x N^2 nodes */
  int64_t nnz_ = 7 * n_ - 6 * N * N;
  if (nnz_ > INT32_MAX) return -1;
  *n = n_;
  *nnz = nnz_;
  return 0;
}

int gen_lap3d7_fill(int64_t N, int32_t* rowptr, int32_t* colind, double* vals) {
  int64_t n_, nnz_;
  if (gen_lap3d7_size(N, &n_, &nnz_)) return -1;
  static const int off[7][3] = {{0, 0, -1}, {0, -1, 0}, {-1, 0, 0}, {0, 0, 0},
                                {1, 0, 0},  {0, 1, 0},  {0, 0, 1}};
  int64_t k = 0;
  rowptr[0] = 0;
  for (int64_t z = 0; z < N; ++z)
    for (int64_t y = 0; y < N; ++y)
      for (int64_t x = 0; x < N; ++x) {
        for (int t = 0; t < 7; ++t) {
          int64_t xx = x + off[t][0], yy = y + off[t][1], zz = z + off[t][2];
          if (xx < 0 || xx >= N || yy < 0 || yy >= N || zz < 0 || zz >= N) continue;
          colind[k] = (int32_t)((zz * N + yy) * N + xx);
          vals[k] = (t == 3) ? 6.0 : -1.0;
          ++k;
        }
        rowptr[(z * N + y) * N + x + 1] = (int32_t)k;
      }
  return 0;
}

/* ------------------------------------------------------------------ */
/* 3-D 27-point variable-coefficient diffusion (weighted graph Laplacian) */
/* ------------------------------------------------------------------ */
/* Every lattice edge {u, u+d}, d one of the 26 neighbour offsets, carries
 * w = s_d * exp(sigma * Z) with s_d = 1 (face), 1/2 (edge), 1/4 (corner)
 * and Z a standard normal drawn per undirected edge.  Edges to nodes outside
 * the N^3 domain exist too (their far end is a Dirichlet ghost).  Row i holds
 * -w for each in-domain neighbour and the sum of all 26 incident weights on
 * the diagonal, so every row is weakly dominant and boundary rows strictly.
 *
 * Edge identity: an undirected edge is named by its endpoint u that has the
 * lexicographically smaller padded position and by the index (0..12) of the
 * "positive" offset d = v - u.  Positions are padded by one layer so that
 * ghost endpoints have indices too: P(x,y,z) = ((z+1)(N+2) + y+1)(N+2) + x+1.
 * The normal deviate of edge (u, dir) is gen_normal(seed, P(u)*13 + dir). */

static int pos_dir_index(int dx, int dy, int dz) {
  /* positive offsets: (dz, dy, dx) > (0, 0, 0) lexicographically */
  int code = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1); /* 0..26, 13 = zero */
  return code - 14; /* 14..26 -> 0..12 */
}

static double edge_weight(int64_t N, uint64_t seed, double sigma,
                          int64_t x, int64_t y, int64_t z, int dx, int dy, int dz) {
  int code = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
  if (code < 13) { /* negative offset: name the edge from the other end */
    x += dx; y += dy; z += dz;
    dx = -dx; dy = -dy; dz = -dz;
  }
  const int64_t M = N + 2;
  const int64_t P = ((z + 1) * M + (y + 1)) * M + (x + 1);
  const int dir = pos_dir_index(dx, dy, dz);
  const int nz = (dx != 0) + (dy != 0) + (dz != 0);
  const double s = (nz == 1) ? 1.0 : (nz == 2) ? 0.5 : 0.25;
  return s * exp(sigma * gen_normal(seed, (uint64_t)P * 13u + (uint64_t)dir));
}

int gen_diff3d27_size(int64_t N, int64_t* n, int64_t* nnz) {
  if (N < 1 || N > 1000) return -1;
  int64_t per_axis = 3 * N - 2; /* sum over x of in-range neighbours in {-1,0,1} */
  int64_t nnz_ = per_axis * per_axis * per_axis;
  if (nnz_ > INT32_MAX) return -1;
  *n = N * N * N;
  *nnz = nnz_;
  return 0;
}

int gen_diff3d27_fill(int64_t N, double sigma, uint64_t seed,
                      int32_t* rowptr, int32_t* colind, double* vals) {
  int64_t n_, nnz_;
  if (gen_diff3d27_size(N, &n_, &nnz_)) return -1;
  if (!(sigma >= 0.0)) return -1;
  int64_t k = 0;
  rowptr[0] = 0;
  for (int64_t z = 0; z < N; ++z)
    for (int64_t y = 0; y < N; ++y)
      for (int64_t x = 0; x < N; ++x) {
        double diag = 0.0;
        int64_t kdiag = -1;
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              int64_t xx = x + dx, yy = y + dy, zz = z + dz;
              int inside = xx >= 0 && xx < N && yy >= 0 && yy < N && zz >= 0 && zz < N;
              if (dx == 0 && dy == 0 && dz == 0) {
                colind[k] = (int32_t)((z * N + y) * N + x);
                kdiag = k++;
                continue;
              }
              double w = edge_weight(N, seed, sigma, x, y, z, dx, dy, dz);
              diag += w;
              if (!inside) continue;
              colind[k] = (int32_t)((zz * N + yy) * N + xx);
              vals[k] = -w;
              ++k;
            }
        vals[kdiag] = diag;
        rowptr[(z * N + y) * N + x + 1] = (int32_t)k;
      }
  return 0;
}

/* ------------------------------------------------------------------ */
/* 2-D rotated-anisotropy diffusion, bilinear (Q1) finite elements      */
/* ------------------------------------------------------------------ */
/* Unit square, (s+2) x (s+2) nodes with spacing h = 1/(s+1); the boundary
 * ring is Dirichlet-eliminated, leaving s x s unknowns (x, y), row y*s + x.
 * Cell (cx, cy), 0 <= cx, cy <= s, spans padded nodes cx..cx+1, cy..cy+1 and
 * carries the tensor K_c = a_c R(theta) diag(1, eps) R(theta)^T with
 * a_c = exp(sigma_a * Z(seed, cy*(s+1) + cx)).  In 2-D the Q1 stiffness on a
 * square is independent of h.  With local node (i, j), i, j in {0, 1}, and
 * s_0 = -1, s_1 = +1, M = [[1/3, 1/6], [1/6, 1/3]] the exact element matrix
 * for K = [[kxx, kxy], [kxy, kyy]] is
 *   Ke[(i,j),(k,l)] = kxx s_i s_k M_jl + kyy s_j s_l M_ik
 *                     + kxy (s_i s_l + s_j s_k) / 4.
 * Entries for a pair of nodes sum their shared cells in increasing cell
 * index, so A is bitwise symmetric.  The stencil is the full 9 points. */

static double q1_ke(int i, int j, int k, int l, double kxx, double kyy, double kxy) {
  const double sg[2] = {-1.0, 1.0};
  const double M[2][2] = {{1.0 / 3.0, 1.0 / 6.0}, {1.0 / 6.0, 1.0 / 3.0}};
  return kxx * sg[i] * sg[k] * M[j][l] + kyy * sg[j] * sg[l] * M[i][k] +
         kxy * (sg[i] * sg[l] + sg[j] * sg[k]) / 4.0;
}

int gen_q1aniso_size(int64_t s, int64_t* n, int64_t* nnz) {
  if (s < 1 || s > 46000) return -1;
  int64_t per_axis = 3 * s - 2;
  *n = s * s;
  *nnz = per_axis * per_axis;
  return 0;
}

int gen_q1aniso_fill(int64_t s, double sigma_a, double theta, double eps, uint64_t seed,
                     int32_t* rowptr, int32_t* colind, double* vals) {
  int64_t n_, nnz_;
  if (gen_q1aniso_size(s, &n_, &nnz_)) return -1;
  if (!(eps > 0.0) || !(sigma_a >= 0.0)) return -1;
  const double c = cos(theta), sn = sin(theta);
  const double kxx = c * c + eps * sn * sn;
  const double kyy = sn * sn + eps * c * c;
  const double kxy = (1.0 - eps) * c * sn;
  int64_t k = 0;
  rowptr[0] = 0;
  for (int64_t y = 0; y < s; ++y)
    for (int64_t x = 0; x < s; ++x) {
      const int64_t px = x + 1, py = y + 1; /* padded node coordinates */
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          int64_t xx = x + dx, yy = y + dy;
          if (xx < 0 || xx >= s || yy < 0 || yy >= s) continue;
          const int64_t qx = px + dx, qy = py + dy;
          double v = 0.0;
          /* cells containing both padded nodes, in increasing cell index */
          for (int64_t cy = py - 1; cy <= py; ++cy)
            for (int64_t cx = px - 1; cx <= px; ++cx) {
              if (qx < cx || qx > cx + 1 || qy < cy || qy > cy + 1) continue;
              const double a = exp(sigma_a * gen_normal(seed, (uint64_t)(cy * (s + 1) + cx)));
              v += a * q1_ke((int)(px - cx), (int)(py - cy), (int)(qx - cx), (int)(qy - cy),
                             kxx, kyy, kxy);
            }
          colind[k] = (int32_t)(yy * s + xx);
          vals[k] = v;
          ++k;
        }
      rowptr[y * s + x + 1] = (int32_t)k;
    }
  return 0;
}

/* ------------------------------------------------------------------ */
/* General sparse SPD matrix: a weighted graph Laplacian with power-law  */
/* degrees, plus a small diagonal shift                                 */
/* ------------------------------------------------------------------ */
/* Row i emits h_i = ceil(d_i / 2) edges, d_i = min(dmax, floor(2 u^(-1/1.6)))
 * (a Pareto tail: most rows have 2-6 neighbours, a few hundreds), to partners
 * j that are local (|j - i| <= 64) with probability 0.7 and uniform over all
 * rows otherwise; edge weight w = 0.5 + u.  Every edge couples both of its
 * rows (A_ij = A_ji = -w, duplicates summed), and A_ii = (1 + s_i) sum_j w_ij
 * with s_i = 10^(-4 + u) (the shift makes the Laplacian definite; a row left
 * without couplings gets A_ii = 1; the diagonal is always stored).  Columns are sorted within each row.  Counter
 * layout of the stream: row i uses counters i * 1024 + c, c < 1024. */
static int gspd_half_degree(int64_t i, int32_t dmax, uint64_t seed) {
  const double u = u01_open0(seed, (uint64_t)i * 1024 + 1023);
  double d = floor(2.0 * pow(u, -1.0 / 1.6));
  if (d > (double)dmax) d = (double)dmax;
  return (int)((d + 1.0) / 2.0);
}

/* partner of edge e of row i (i itself means no edge) */
static int64_t gspd_partner(int64_t i, int e, int64_t n, uint64_t seed) {
  const uint64_t c = (uint64_t)i * 1024 + 3 * (uint64_t)e;
  int64_t j;
  if (u01(seed, c) < 0.7)
    j = i + (int64_t)floor((2.0 * u01(seed, c + 1) - 1.0) * 64.5);
  else
    j = (int64_t)floor(u01(seed, c + 1) * (double)n);
  return (j < 0 || j >= n) ? i : j;
}

static int64_t graph_spd_build(int64_t n, int32_t dmax, uint64_t seed, int32_t* rowptr, int32_t* colind,
                               double* vals) {
  if (n <= 0 || n >= INT32_MAX || dmax < 2 || dmax > 600) return -1;
  int32_t* cnt = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  if (!cnt) return -1;
  /* pass 1: row lengths before merging */
  for (int64_t i = 0; i < n; ++i) {
    const int h = gspd_half_degree(i, dmax, seed);
    for (int e = 0; e < h; ++e) {
      const int64_t j = gspd_partner(i, e, n, seed);
      if (j == i) continue;
      ++cnt[i];
      ++cnt[j];
    }
  }
  int64_t* start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  if (!start) { free(cnt); return -1; }
  start[0] = 0;
  for (int64_t i = 0; i < n; ++i) start[i + 1] = start[i] + cnt[i] + 1; /* + the diagonal */
  const int64_t total = start[n];
  int32_t* col = (int32_t*)malloc(sizeof(int32_t) * (size_t)total);
  double* w = (double*)malloc(sizeof(double) * (size_t)total);
  if (!col || !w) { free(cnt); free(start); free(col); free(w); return -1; }
  /* pass 2: both directions of every edge */
  for (int64_t i = 0; i < n; ++i) cnt[i] = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int h = gspd_half_degree(i, dmax, seed);
    for (int e = 0; e < h; ++e) {
      const int64_t j = gspd_partner(i, e, n, seed);
      if (j == i) continue;
      const double we = 0.5 + u01(seed, (uint64_t)i * 1024 + 3 * (uint64_t)e + 2);
      int64_t p = start[i] + cnt[i]++;
      col[p] = (int32_t)j;
      w[p] = we;
      p = start[j] + cnt[j]++;
      col[p] = (int32_t)i;
      w[p] = we;
    }
  }
  /* per row: the diagonal slot, sort by column, merge duplicates, emit */
  int64_t nnz = 0;
  if (rowptr) rowptr[0] = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t a = start[i];
    int64_t e = a + cnt[i];
    col[e] = (int32_t)i;
    w[e] = 0.0;
    ++e;
    for (int64_t k = a + 1; k < e; ++k) { /* insertion sort by column */
      const int32_t ck = col[k];
      const double wk = w[k];
      int64_t m = k - 1;
      while (m >= a && col[m] > ck) {
        col[m + 1] = col[m];
        w[m + 1] = w[m];
        --m;
      }
      col[m + 1] = ck;
      w[m + 1] = wk;
    }
    double wsum = 0.0;
    for (int64_t k = a; k < e; ++k) wsum += w[k];
    const double shift = pow(10.0, -4.0 + u01(seed, (uint64_t)i * 1024 + 1022));
    for (int64_t k = a; k < e;) {
      int64_t m = k;
      double ws = 0.0;
      while (m < e && col[m] == col[k]) ws += w[m++];
      if (colind) {
        colind[nnz] = col[k];
        vals[nnz] = col[k] == (int32_t)i ? (wsum > 0.0 ? (1.0 + shift) * wsum : 1.0) : -ws;
      }
      ++nnz;
      k = m;
    }
    if (rowptr) rowptr[i + 1] = (int32_t)nnz;
    if (nnz >= INT32_MAX) { nnz = -1; break; }
  }
  free(cnt);
  free(start);
  free(col);
  free(w);
  return nnz;
}

int gen_graph_spd_size(int64_t n, int32_t dmax, uint64_t seed, int64_t* n_out, int64_t* nnz) {
  const int64_t z = graph_spd_build(n, dmax, seed, NULL, NULL, NULL);
  if (z < 0) return -1;
  *n_out = n;
  *nnz = z;
  return 0;
}

int gen_graph_spd_fill(int64_t n, int32_t dmax, uint64_t seed, int32_t* rowptr, int32_t* colind,
                       double* vals) {
  return graph_spd_build(n, dmax, seed, rowptr, colind, vals) < 0 ? -1 : 0;
}
