// tf_adjoint.cu -- discrete adjoint of the fixed-iteration Newton--ADI time
// step (reverse of the unrolled iteration of Sec. Numerical Method):
//
//   b = u^n - (1-theta) dt D(u^n),  u_0 = u^n,
//   A_x(u_k) w_k = -G(u_k),  A_y(u_k) v_k = w_k,  u_{k+1} = u_k + v_k,
//   G(u) = u + theta dt D(u) - b,  A = I + theta dt J (x lines, then y lines).
//
// Given the cotangent g of u_K, the reverse sweep (k = K-1 .. 0) is
//   lambda_y = A_y(u_k)^-T ubar                 (transposed y-line solves)
//   ubar    -= [d_u (A_y(u) v_k)]^T lambda_y    (coefficient dependence)
//   lambda_x = A_x(u_k)^-T lambda_y             (transposed x-line solves)
//   ubar    -= [d_u (A_x(u) w_k)]^T lambda_x
//   ubar    -= lambda_x + theta dt D'(u_k)^T lambda_x,   bbar += lambda_x
// and finally ubar += bbar - (1-theta) dt D'(u^n)^T bbar; the kappa
// cotangent collects the same terms' kappa derivatives.
//
// Derivatives: forward-mode dual numbers over per-iterate tables (the
// mobilities with two derivatives and the Laplacian, formed once per
// iterate), so a seeded evaluation only propagates the seeded cell's known
// partials.  The value of D at a cell depends
// on u within the 13-cell diamond |dx| + |dy| <= 2 around it, and a row of
// A_x(u) w on u within the box |dx| <= 2, |dy| <= 1 (A_y: transposed).  So
// the transposed product at cell j is a gather over the cells c whose
// dependence set holds j: one thread per j evaluates each such F_c with u_j
// seeded and sums lambda_c dF_c/du_j.  No atomics; every sum runs in a fixed
// order.  FP64 throughout; the power-law and linear models.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "tf_internal.h"

namespace {

struct Dual {
  double v, d;
};
__device__ __forceinline__ Dual mk(double v, double d = 0.0) { return Dual{v, d}; }
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return Dual{a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return Dual{a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return Dual{a.v * b.v, a.v * b.d + a.d * b.v}; }
__device__ __forceinline__ Dual operator*(double s, Dual a) { return Dual{s * a.v, s * a.d}; }

struct AdjK {
  int nx, ny, model, n, m;
  double ds, inv_ds, C, b, c0, c1, kappa, tdt;  // tdt = theta dt
};

// Per-cell values of the iterate, formed once per iterate (FP64):
// f0, f1, f0', f1', f0'', f1'' (Sec. Thin Film Models: f0 = C h^3,
// f1 = h^3 Pi'(h), Pi = kappa[(b/h)^n - (b/h)^m]) and the Laplacian.
struct Tables {
  double *f0, *f1, *d0, *d1, *e0, *e1, *lap;
};

__global__ void k_tables(AdjK M, const double* __restrict__ u, Tables T) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= M.nx) return;
  const size_t c = (size_t)j * M.nx + i;
  const double h = u[c];
  if (M.model == TF_MODEL_LINEAR) {
    T.f0[c] = M.c0;
    T.f1[c] = M.c1;
    T.d0[c] = T.d1[c] = T.e0[c] = T.e1[c] = 0.0;
  } else {
    // Pi' = kappa (m r^m - n r^n)/h, Pi'' = kappa (n(n+1) r^n - m(m+1) r^m)/h^2,
    // Pi''' = kappa (m(m+1)(m+2) r^m - n(n+1)(n+2) r^n)/h^3, r = b/h
    const double ih = 1.0 / h, r = M.b * ih;
    double rm = 1.0, rn = 1.0;
    for (int q = 0; q < M.m; ++q) rm *= r;
    for (int q = 0; q < M.n; ++q) rn *= r;
    const double n = M.n, m = M.m;
    const double p1 = M.kappa * (m * rm - n * rn) * ih;
    const double p2 = M.kappa * (n * (n + 1.0) * rn - m * (m + 1.0) * rm) * ih * ih;
    const double p3 = M.kappa * (m * (m + 1.0) * (m + 2.0) * rm - n * (n + 1.0) * (n + 2.0) * rn) * ih * ih * ih;
    const double h2 = h * h, h3 = h2 * h;
    T.f0[c] = M.C * h3;
    T.f1[c] = h3 * p1;
    T.d0[c] = 3.0 * M.C * h2;
    T.d1[c] = 3.0 * h2 * p1 + h3 * p2;
    T.e0[c] = 6.0 * M.C * h;
    T.e1[c] = 6.0 * h * p1 + 6.0 * h2 * p2 + h3 * p3;
  }
  double sl = 0.0;
  if (i + 1 < M.nx) sl += u[c + 1] - h;
  if (i > 0) sl += u[c - 1] - h;
  if (j + 1 < M.ny) sl += u[c + M.nx] - h;
  if (j > 0) sl += u[c - M.nx] - h;
  T.lap[c] = sl * M.inv_ds * M.inv_ds;
}

struct Mob {
  Dual f0, f1, d0, d1;
};

// The film seen by one evaluation: values from the tables, derivatives
// with respect to the one seeded quantity -- u at cell (pi, pj) (pi < 0:
// none) or kappa (kseed; f1 and f1' are linear in kappa).
struct Film {
  const double* u;
  Tables T;
  int nx, ny, pi, pj;
  bool kseed;
  double inv_kappa, inv_ds2;
  __device__ __forceinline__ bool seeded(int i, int j) const { return i == pi && j == pj; }
  __device__ __forceinline__ Dual at(int i, int j) const {
    return Dual{u[(size_t)j * nx + i], seeded(i, j) ? 1.0 : 0.0};
  }
  __device__ __forceinline__ Mob mob(int i, int j) const {
    const size_t c = (size_t)j * nx + i;
    const double f0 = T.f0[c], f1 = T.f1[c], d0 = T.d0[c], d1 = T.d1[c];
    if (kseed) return Mob{mk(f0), mk(f1, f1 * inv_kappa), mk(d0), mk(d1, d1 * inv_kappa)};
    if (!seeded(i, j)) return Mob{mk(f0), mk(f1), mk(d0), mk(d1)};
    return Mob{mk(f0, d0), mk(f1, d1), mk(d0, T.e0[c]), mk(d1, T.e1[c])};
  }
  // Five-point Laplacian with even reflection; its derivative with respect
  // to the seeded cell is -(neighbours)/ds^2 at that cell, 1/ds^2 next to it.
  __device__ __forceinline__ Dual lap(int i, int j) const {
    const double v = T.lap[(size_t)j * nx + i];
    if (pi < 0) return mk(v);
    const int di = pi - i, dj = pj - j;
    if (di == 0 && dj == 0) {
      const int cnt = (i + 1 < nx) + (i > 0) + (j + 1 < ny) + (j > 0);
      return mk(v, -(double)cnt * inv_ds2);
    }
    const int ad = (di < 0 ? -di : di) + (dj < 0 ? -dj : dj);
    return mk(v, ad == 1 ? inv_ds2 : 0.0);
  }
};

// Flux through the face from cell p to its +x or +y neighbour q:
// F = fbar0 (L_q - L_p)/ds + fbar1 (u_q - u_p)/ds, fbar the two cells' mean.
__device__ Dual face_flux(const AdjK& M, Dual up, Dual uq, Dual lp, Dual lq, const Mob& mp, const Mob& mq) {
  return (0.5 * M.inv_ds) * ((mp.f0 + mq.f0) * (lq - lp) + (mp.f1 + mq.f1) * (uq - up));
}

// D at cell (i, j) (eq. GovEqnCell2, zero wall fluxes).
__device__ Dual D_cell(const AdjK& M, const Film& F, int i, int j) {
  const Dual uc = F.at(i, j), lc = F.lap(i, j);
  const Mob mc = F.mob(i, j);
  Dual acc = mk(0.0);
  if (i + 1 < M.nx) acc = acc + face_flux(M, uc, F.at(i + 1, j), lc, F.lap(i + 1, j), mc, F.mob(i + 1, j));
  if (i > 0) acc = acc - face_flux(M, F.at(i - 1, j), uc, F.lap(i - 1, j), lc, F.mob(i - 1, j), mc);
  if (j + 1 < M.ny) acc = acc + face_flux(M, uc, F.at(i, j + 1), lc, F.lap(i, j + 1), mc, F.mob(i, j + 1));
  if (j > 0) acc = acc - face_flux(M, F.at(i, j - 1), uc, F.lap(i, j - 1), lc, F.mob(i, j - 1), mc);
  return M.inv_ds * acc;
}

// d(along-line second difference at line cell c)/d(u at line cell col),
// reflection at the ends of a line of n cells, times ds^2.
__device__ __forceinline__ double dlap_line(int c, int col, int n) {
  if (col == c + 1) return c < n - 1 ? 1.0 : 0.0;
  if (col == c - 1) return c > 0 ? 1.0 : 0.0;
  if (col == c) return -(double)((c < n - 1) + (c > 0));
  return 0.0;
}

// Row of I + theta dt J along a line (DIR 0: x, the line is row j; DIR 1: y,
// column i) at the line cell t = i or j: band[d] is the coefficient of line
// cell t + d - 2.  Face between line cells p and q = p + 1: the flux
// derivative has f0'/2 gL and f1'/2 gU on p and q (gL = (L_q - L_p)/ds with
// the full Laplacian, gU = (u_q - u_p)/ds), fbar0 (dLline_q - dLline_p)/ds
// over columns p-1..p+2, and -+fbar1/ds on p, q; row p gets +theta dt dF/ds,
// row q -theta dt dF/ds.
template <int DIR>
__device__ void row_band(const AdjK& M, const Film& F, int i, int j, Dual (&band)[5]) {
  const int n = DIR == 0 ? M.nx : M.ny, t = DIR == 0 ? i : j;
  for (int d = 0; d < 5; ++d) band[d] = mk(d == 2 ? 1.0 : 0.0);
  auto cell = [&](int s, int& ci, int& cj) {
    ci = DIR == 0 ? s : i;
    cj = DIR == 0 ? j : s;
  };
  for (int side = 0; side < 2; ++side) {
    const int p = side == 0 ? t - 1 : t, q = p + 1;
    if (p < 0 || q >= n) continue;
    int pi, pj, qi, qj;
    cell(p, pi, pj);
    cell(q, qi, qj);
    const Dual up = F.at(pi, pj), uq = F.at(qi, qj);
    const Dual lp = F.lap(pi, pj), lq = F.lap(qi, qj);
    const Mob mp = F.mob(pi, pj), mq = F.mob(qi, qj);
    const Dual fb0 = 0.5 * (mp.f0 + mq.f0), fb1 = 0.5 * (mp.f1 + mq.f1);
    const Dual gL = M.inv_ds * (lq - lp), gU = M.inv_ds * (uq - up);
    const double sgn = side == 0 ? -1.0 : 1.0;  // row t is q (side 0) or p (side 1)
    const double coef = sgn * M.tdt * M.inv_ds;
    for (int a = 0; a < 4; ++a) {
      const int col = p - 1 + a;
      if (col < 0 || col >= n) continue;
      const double dl = (dlap_line(q, col, n) - dlap_line(p, col, n)) * M.inv_ds * M.inv_ds * M.inv_ds;
      Dual v = dl * fb0;
      if (col == p) v = v + 0.5 * (mp.d0 * gL) + 0.5 * (mp.d1 * gU) - M.inv_ds * fb1;
      if (col == q) v = v + 0.5 * (mq.d0 * gL) + 0.5 * (mq.d1 * gU) + M.inv_ds * fb1;
      band[col - t + 2] = band[col - t + 2] + coef * v;
    }
  }
}

// (A(u) w) at cell (i, j) along direction DIR.
template <int DIR>
__device__ Dual row_times(const AdjK& M, const Film& F, const double* __restrict__ w, int i, int j) {
  Dual band[5];
  row_band<DIR>(M, F, i, j, band);
  const int n = DIR == 0 ? M.nx : M.ny, t = DIR == 0 ? i : j;
  Dual acc = mk(0.0);
  for (int d = 0; d < 5; ++d) {
    const int s = t + d - 2;
    if (s < 0 || s >= n) continue;
    const double ws = DIR == 0 ? w[(size_t)j * M.nx + s] : w[(size_t)s * M.nx + i];
    acc = acc + ws * band[d];
  }
  return acc;
}

__device__ __forceinline__ Film make_film(const AdjK& M, const double* u, const Tables& T, int pi, int pj,
                                          bool kseed) {
  return Film{u, T, M.nx, M.ny, pi, pj, kseed, M.model == TF_MODEL_LINEAR ? 0.0 : 1.0 / M.kappa,
              M.inv_ds * M.inv_ds};
}

// ubar_j += scale * sum_{c: |c - j|_1 <= 2} lambda_c dD_c/du_j
__global__ void k_adj_D(AdjK M, const double* __restrict__ u, Tables T, const double* __restrict__ lam,
                        double scale, double* __restrict__ ubar) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= M.nx) return;
  const Film F = make_film(M, u, T, i, j, false);
  double acc = 0.0;
  for (int dy = -2; dy <= 2; ++dy) {
    const int cj = j + dy;
    if (cj < 0 || cj >= M.ny) continue;
    const int r = 2 - (dy < 0 ? -dy : dy);
    for (int dx = -r; dx <= r; ++dx) {
      const int ci = i + dx;
      if (ci < 0 || ci >= M.nx) continue;
      acc += lam[(size_t)cj * M.nx + ci] * D_cell(M, F, ci, cj).d;
    }
  }
  ubar[(size_t)j * M.nx + i] += scale * acc;
}

// ubar_j += scale * sum_{c in box(j)} lambda_c d(A(u) w)_c/du_j, box |dx| <= 2,
// |dy| <= 1 along x (transposed along y).
template <int DIR>
__global__ void k_adj_line(AdjK M, const double* __restrict__ u, Tables T, const double* __restrict__ w,
                           const double* __restrict__ lam, double scale, double* __restrict__ ubar) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= M.nx) return;
  const Film F = make_film(M, u, T, i, j, false);
  const int rx = DIR == 0 ? 2 : 1, ry = DIR == 0 ? 1 : 2;
  double acc = 0.0;
  for (int dy = -ry; dy <= ry; ++dy) {
    const int cj = j + dy;
    if (cj < 0 || cj >= M.ny) continue;
    for (int dx = -rx; dx <= rx; ++dx) {
      const int ci = i + dx;
      if (ci < 0 || ci >= M.nx) continue;
      acc += lam[(size_t)cj * M.nx + ci] * row_times<DIR>(M, F, w, ci, cj).d;
    }
  }
  ubar[(size_t)j * M.nx + i] += scale * acc;
}

// Per-block partial sums of lambda_c dF_c/dkappa for F = D (kind 0), A_x w
// (kind 1) or A_y w (kind 2): blocks of 256 cells in row-major order, summed
// by a fixed tree.
constexpr int kKapThreads = 256;
__global__ void __launch_bounds__(kKapThreads) k_adj_kappa(AdjK M, int kind, const double* __restrict__ u,
                                                            Tables T, const double* __restrict__ w,
                                                            const double* __restrict__ lam,
                                                            double* __restrict__ part) {
  __shared__ double s[kKapThreads];
  const size_t N = (size_t)M.nx * M.ny;
  const size_t c = (size_t)blockIdx.x * kKapThreads + threadIdx.x;
  double v = 0.0;
  if (c < N) {
    const int i = (int)(c % M.nx), j = (int)(c / M.nx);
    const Film F = make_film(M, u, T, -1, -1, true);
    const Dual val = kind == 0 ? D_cell(M, F, i, j)
                               : (kind == 1 ? row_times<0>(M, F, w, i, j) : row_times<1>(M, F, w, i, j));
    v = lam[c] * val.d;
  }
  s[threadIdx.x] = v;
  __syncthreads();
  for (int h = kKapThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// Band of A along DIR at every cell: band[d * N + c] (values only).
template <int DIR>
__global__ void k_band(AdjK M, const double* __restrict__ u, Tables T, double* __restrict__ band) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= M.nx) return;
  const Film F = make_film(M, u, T, -1, -1, false);
  Dual b[5];
  row_band<DIR>(M, F, i, j, b);
  const size_t N = (size_t)M.nx * M.ny, c = (size_t)j * M.nx + i;
  for (int d = 0; d < 5; ++d) band[d * N + c] = b[d].v;
}

// Transposed pentadiagonal solves A^T x = r along every line of direction
// DIR, one thread per line, elimination without pivoting (bandwidth 2) and
// back substitution.  Row t of A^T holds A[t+d-2][t] = band[4-d] of row
// t+d-2.  scratch: 4 values per cell (eliminated row and right side).
template <int DIR>
__global__ void k_solve_t(int nx, int ny, const double* __restrict__ band, const double* __restrict__ r,
                          double* __restrict__ x, double* __restrict__ scratch) {
  const int line = blockIdx.x * blockDim.x + threadIdx.x;
  const int nlines = DIR == 0 ? ny : nx, n = DIR == 0 ? nx : ny;
  if (line >= nlines) return;
  const size_t N = (size_t)nx * ny;
  auto idx = [&](int t) -> size_t { return DIR == 0 ? (size_t)line * nx + t : (size_t)t * nx + line; };
  auto B = [&](int row, int d) -> double { return (row < 0 || row >= n) ? 0.0 : band[d * N + idx(row)]; };
  // transposed row t: (lo2, lo1, dg, up1, up2)
  auto trow = [&](int t, double& lo2, double& lo1, double& dg, double& up1, double& up2) {
    lo2 = B(t - 2, 4);
    lo1 = B(t - 1, 3);
    dg = B(t, 2);
    up1 = B(t + 1, 1);
    up2 = B(t + 2, 0);
  };
  double* sd = scratch;          // reciprocal of the eliminated diagonal
  double* s1 = scratch + N;      // eliminated first super-diagonal
  double* s2 = scratch + 2 * N;  // second super-diagonal
  double* sy = scratch + 3 * N;  // eliminated right side
  // window: rows k (a*), k+1 (b*), k+2 (c*); rows k+2..k+5 are loaded four
  // steps ahead into a ring (slot = row mod 4) so that the loads overlap the
  // elimination chain
  double a_lo2, a_lo1, a_dg, a_u1, a_u2, a_y;
  double b_lo2 = 0.0, b_lo1 = 0.0, b_dg = 1.0, b_u1 = 0.0, b_u2 = 0.0, b_y = 0.0;
  double c_lo2 = 0.0, c_lo1 = 0.0, c_dg = 1.0, c_u1 = 0.0, c_u2 = 0.0, c_y = 0.0;
  double p_lo2[4], p_lo1[4], p_dg[4], p_u1[4], p_u2[4], p_y[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    p_lo2[q] = p_lo1[q] = p_u1[q] = p_u2[q] = p_y[q] = 0.0;
    p_dg[q] = 1.0;
  }
  trow(0, a_lo2, a_lo1, a_dg, a_u1, a_u2);
  a_y = r[idx(0)];
  if (n > 1) {
    trow(1, b_lo2, b_lo1, b_dg, b_u1, b_u2);
    b_y = r[idx(1)];
  }
#pragma unroll
  for (int q = 2; q < 6; ++q) {
    if (q < n) {
      trow(q, p_lo2[q & 3], p_lo1[q & 3], p_dg[q & 3], p_u1[q & 3], p_u2[q & 3]);
      p_y[q & 3] = r[idx(q)];
    }
  }
  for (int k0 = 0; k0 < n; k0 += 4) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = k0 + q, sl = (q + 2) & 3;  // ring slot of row k + 2
      if (k < n) {
        if (k + 2 < n) {
          c_lo2 = p_lo2[sl];
          c_lo1 = p_lo1[sl];
          c_dg = p_dg[sl];
          c_u1 = p_u1[sl];
          c_u2 = p_u2[sl];
          c_y = p_y[sl];
        }
        if (k + 6 < n) {
          trow(k + 6, p_lo2[sl], p_lo1[sl], p_dg[sl], p_u1[sl], p_u2[sl]);
          p_y[sl] = r[idx(k + 6)];
        }
        const double inv = 1.0 / a_dg;
        if (k + 1 < n) {
          const double l = b_lo1 * inv;
          b_dg -= l * a_u1;
          b_u1 -= l * a_u2;
          b_y -= l * a_y;
        }
        if (k + 2 < n) {
          const double l = c_lo2 * inv;
          c_lo1 -= l * a_u1;
          c_dg -= l * a_u2;
          c_y -= l * a_y;
        }
        const size_t ck = idx(k);
        sd[ck] = inv;
        s1[ck] = a_u1;
        s2[ck] = a_u2;
        sy[ck] = a_y;
        // shift the window
        a_lo2 = b_lo2;
        a_lo1 = b_lo1;
        a_dg = b_dg;
        a_u1 = b_u1;
        a_u2 = b_u2;
        a_y = b_y;
        b_lo2 = c_lo2;
        b_lo1 = c_lo1;
        b_dg = c_dg;
        b_u1 = c_u1;
        b_u2 = c_u2;
        b_y = c_y;
      }
    }
  }
  double x1 = 0.0, x2 = 0.0;  // x_{k+1}, x_{k+2}
#pragma unroll 4
  for (int k = n - 1; k >= 0; --k) {
    const size_t ck = idx(k);
    const double xv = (sy[ck] - s1[ck] * x1 - s2[ck] * x2) * sd[ck];
    x[ck] = xv;
    x2 = x1;
    x1 = xv;
  }
}

__global__ void k_axpy(size_t N, double a, const double* __restrict__ x, double* __restrict__ y) {
  const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < N) y[c] += a * x[c];
}

// Kernel groups timed by tf_adjoint_step (CUDA events on the context's
// stream, summed over the call).
enum { kGForward, kGBand, kGSolve, kGLineX, kGLineY, kGD, kGKappa, kGroups };

struct GroupTimer {
  cudaStream_t st;
  std::vector<cudaEvent_t> ev;
  std::vector<int> group;
  cudaError_t err = cudaSuccess;
  int begin(int g) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) err = cudaErrorUnknown;
    ev.push_back(a);
    ev.push_back(b);
    group.push_back(g);
    cudaEventRecord(a, st);
    return (int)group.size() - 1;
  }
  void end(int k) { cudaEventRecord(ev[2 * k + 1], st); }
  void collect(double* ms) {
    for (int g = 0; g < kGroups; ++g) ms[g] = 0.0;
    for (size_t k = 0; k < group.size(); ++k) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, ev[2 * k], ev[2 * k + 1]) == cudaSuccess) ms[group[k]] += t;
    }
  }
  ~GroupTimer() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

double g_adj_ms[kGroups];  // last call's group times (the library's callers
                           // serialise adjoint calls per process for timing)

}  // namespace

extern "C" int tf_adjoint_timing(double* ms, int n) {
  if (!ms || n < 1) return TF_ERR_ARG;
  for (int g = 0; g < n && g < kGroups; ++g) ms[g] = g_adj_ms[g];
  return TF_OK;
}

extern "C" int tf_adjoint_step(tf_ctx* c, const double* h_old, double dt, int K, const double* g,
                               double* h_new, double* g_h, double* g_kappa, double* g_theta) {
  if (!c || !h_old || !g || !g_h || K < 1 || K > 64 || !(dt > 0.0) || !isfinite(dt)) return TF_ERR_ARG;
  if (c->p.precision != TF_FP64) return TF_ERR_ARG;
  if (c->p.model != TF_MODEL_POWERLAW && c->p.model != TF_MODEL_LINEAR) return TF_ERR_ARG;
  if (g_h == h_old || g_h == g || (h_new && (h_new == h_old || h_new == g_h))) return TF_ERR_ARG;
  const int nx = c->p.nx, ny = c->p.ny;
  const size_t N = c->N;
  cudaStream_t st = c->stream;
  const int kb = (int)((N + kKapThreads - 1) / kKapThreads);
  // workspace: u_1..u_K, w_0..w_{K-1}, v_0..v_{K-1}, band (5), lam_y, lam_x,
  // bbar, scratch (4), kappa partials
  const size_t grids = (size_t)3 * K + 5 + 3 + 4 + 7;
  const size_t bytes = grids * N * sizeof(double) + (size_t)kb * sizeof(double) * 8;
  if (c->adj_bytes < bytes) {
    if (c->adj_ws) cudaFree(c->adj_ws);
    c->adj_ws = nullptr;
    c->adj_bytes = 0;
    if (cudaMalloc(&c->adj_ws, bytes) != cudaSuccess) return TF_ERR_NOMEM;
    c->adj_bytes = bytes;
  }
  double* base = (double*)c->adj_ws;
  std::vector<double*> U(K + 1), W(K), V(K);
  U[0] = const_cast<double*>(h_old);
  size_t off = 0;
  for (int k = 1; k <= K; ++k, off += N) U[k] = base + off;
  for (int k = 0; k < K; ++k, off += N) W[k] = base + off;
  for (int k = 0; k < K; ++k, off += N) V[k] = base + off;
  double* band = base + off;
  off += 5 * N;
  double* lam_y = base + off;
  off += N;
  double* lam_x = base + off;
  off += N;
  double* bbar = base + off;
  off += N;
  double* scratch = base + off;
  off += 4 * N;
  Tables Tb;
  Tb.f0 = base + off;
  Tb.f1 = Tb.f0 + N;
  Tb.d0 = Tb.f1 + N;
  Tb.d1 = Tb.d0 + N;
  Tb.e0 = Tb.d1 + N;
  Tb.e1 = Tb.e0 + N;
  Tb.lap = Tb.e1 + N;
  off += 7 * N;
  double* part = base + off;  // 8 kinds of partials, kb each

  GroupTimer T;
  T.st = st;
  // forward: K iterations of the FP64 path, keeping u_k, w_k, v_k
  const int tf0 = T.begin(kGForward);
  for (int k = 0; k < K; ++k) {
    tf_step_info info;
    const int r = tf_newton_iteration(c, U[k], h_old, dt, W[k], V[k], U[k + 1], &info);
    if (r < 0) return r;
  }
  T.end(tf0);
  if (h_new && cudaMemcpyAsync(h_new, U[K], N * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return TF_ERR_CUDA;

  AdjK M;
  M.nx = nx;
  M.ny = ny;
  M.model = c->p.model;
  M.n = c->p.n;
  M.m = c->p.m;
  M.ds = c->p.ds;
  M.inv_ds = 1.0 / c->p.ds;
  M.C = c->p.cap_C;
  M.b = c->p.b;
  M.c0 = c->p.c0;
  M.c1 = c->p.c1;
  M.kappa = c->kappa;
  const double theta = c->p.theta;
  M.tdt = theta * dt;

  const dim3 g2((nx + 127) / 128, ny), b2(128);
  // one thread per line, 32 per block so that the lines spread over many SMs
  const int nl_x = (ny + 31) / 32, nl_y = (nx + 31) / 32;
  const int nb = (int)((N + 255) / 256);
  std::vector<double> hp((size_t)kb);
  double kbar = 0.0;
  // kappa terms are summed on the host after each launch (fixed order)
  auto kappa_term = [&](int kind, const double* u, const double* w, const double* lam, double scale) -> int {
    const int tk = T.begin(kGKappa);
    k_adj_kappa<<<kb, kKapThreads, 0, st>>>(M, kind, u, Tb, w, lam, part);
    T.end(tk);
    if (cudaMemcpyAsync(hp.data(), part, kb * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return TF_ERR_CUDA;
    double s = 0.0;
    for (int q = 0; q < kb; ++q) s += hp[q];
    kbar += scale * s;
    return TF_OK;
  };
  const bool kappa_on = M.model == TF_MODEL_POWERLAW;

  if (cudaMemcpyAsync(g_h, g, N * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(bbar, 0, N * sizeof(double), st) != cudaSuccess)
    return TF_ERR_CUDA;
  for (int k = K - 1; k >= 0; --k) {
    const double* uk = U[k];
    // v_k = A_y(u_k)^-1 w_k
    int t = T.begin(kGBand);
    k_tables<<<g2, b2, 0, st>>>(M, uk, Tb);
    k_band<1><<<g2, b2, 0, st>>>(M, uk, Tb, band);
    T.end(t);
    t = T.begin(kGSolve);
    k_solve_t<1><<<nl_y, 32, 0, st>>>(nx, ny, band, g_h, lam_y, scratch);
    T.end(t);
    t = T.begin(kGLineY);
    k_adj_line<1><<<g2, b2, 0, st>>>(M, uk, Tb, V[k], lam_y, -1.0, g_h);
    T.end(t);
    if (kappa_on && kappa_term(2, uk, V[k], lam_y, -1.0)) return TF_ERR_CUDA;
    // w_k = A_x(u_k)^-1 (-G(u_k))
    t = T.begin(kGBand);
    k_band<0><<<g2, b2, 0, st>>>(M, uk, Tb, band);
    T.end(t);
    t = T.begin(kGSolve);
    k_solve_t<0><<<nl_x, 32, 0, st>>>(nx, ny, band, lam_y, lam_x, scratch);
    T.end(t);
    t = T.begin(kGLineX);
    k_adj_line<0><<<g2, b2, 0, st>>>(M, uk, Tb, W[k], lam_x, -1.0, g_h);
    T.end(t);
    if (kappa_on && kappa_term(1, uk, W[k], lam_x, -1.0)) return TF_ERR_CUDA;
    // -G(u_k) = -u_k - theta dt D(u_k) + b
    k_axpy<<<nb, 256, 0, st>>>(N, -1.0, lam_x, g_h);
    k_axpy<<<nb, 256, 0, st>>>(N, 1.0, lam_x, bbar);
    t = T.begin(kGD);
    k_adj_D<<<g2, b2, 0, st>>>(M, uk, Tb, lam_x, -M.tdt, g_h);
    T.end(t);
    if (kappa_on && kappa_term(0, uk, nullptr, lam_x, -M.tdt)) return TF_ERR_CUDA;
  }
  // b = u^n - (1-theta) dt D(u^n)
  const double ex = (1.0 - theta) * dt;
  k_axpy<<<nb, 256, 0, st>>>(N, 1.0, bbar, g_h);
  {
    const int t = T.begin(kGD);
    k_adj_D<<<g2, b2, 0, st>>>(M, h_old, Tb, bbar, -ex, g_h);  // tables of u_0 = h_old
    T.end(t);
  }
  if (kappa_on && kappa_term(0, h_old, nullptr, bbar, -ex)) return TF_ERR_CUDA;
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return TF_ERR_CUDA;
  if (T.err != cudaSuccess) return TF_ERR_CUDA;
  T.collect(g_adj_ms);
  if (g_kappa) *g_kappa = kbar;
  if (g_theta) {
    // kappa = (1 - cos theta_c)/(b M) when derived from the contact angle
    double dk = 0.0;
    if (c->p.kappa <= 0.0 && M.model == TF_MODEL_POWERLAW) {
      const double Mf = (double)(c->p.n - c->p.m) / ((double)(c->p.m - 1) * (double)(c->p.n - 1));
      dk = sin(c->p.contact_angle) / (c->p.b * Mf);
    }
    *g_theta = kbar * dk;
  }
  return TF_OK;
}
