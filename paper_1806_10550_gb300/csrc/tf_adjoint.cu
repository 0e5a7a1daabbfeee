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
// Derivatives: hand-derived face by face from per-iterate tables (the
// mobilities with two derivatives and the Laplacian, formed once per
// iterate); see the comment above k_vjp_D.  Every face term depends on u
// directly at its two cells and through the Laplacian at those cells, so
// each transposed product is two gathers: one thread per cell over the
// faces that touch it, then the transposed five-point Laplacian of the
// collected Laplacian cotangents.  No atomics; every sum runs in a fixed
// order.  FP64 throughout; the power-law and linear models.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <thread>
#include <utility>
#include <vector>

#include "tf_internal.h"

namespace {

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
__device__ void row_band(const AdjK& M, const double* __restrict__ u, const Tables& T, int i, int j,
                         double (&band)[5]) {
  const int n = DIR == 0 ? M.nx : M.ny, t = DIR == 0 ? i : j;
  const size_t c = (size_t)j * M.nx + i, step = DIR == 0 ? 1 : (size_t)M.nx;
  for (int d = 0; d < 5; ++d) band[d] = d == 2 ? 1.0 : 0.0;
  for (int side = 0; side < 2; ++side) {
    const int p = side == 0 ? t - 1 : t, q = p + 1;
    if (p < 0 || q >= n) continue;
    const size_t cp = side == 0 ? c - step : c, cq = cp + step;
    const double fb0 = 0.5 * (T.f0[cp] + T.f0[cq]), fb1 = 0.5 * (T.f1[cp] + T.f1[cq]);
    const double gL = M.inv_ds * (T.lap[cq] - T.lap[cp]), gU = M.inv_ds * (u[cq] - u[cp]);
    const double sgn = side == 0 ? -1.0 : 1.0;  // row t is q (side 0) or p (side 1)
    const double coef = sgn * M.tdt * M.inv_ds;
    for (int a = 0; a < 4; ++a) {
      const int col = p - 1 + a;
      if (col < 0 || col >= n) continue;
      const double dl = (dlap_line(q, col, n) - dlap_line(p, col, n)) * M.inv_ds * M.inv_ds * M.inv_ds;
      double v = dl * fb0;
      if (col == p) v += 0.5 * T.d0[cp] * gL + 0.5 * T.d1[cp] * gU - M.inv_ds * fb1;
      if (col == q) v += 0.5 * T.d0[cq] * gL + 0.5 * T.d1[cq] * gU + M.inv_ds * fb1;
      band[col - t + 2] += coef * v;
    }
  }
}

// ---- transposed derivative products, hand-derived (two passes) ----------
// Face between cells p and q (q the +x or +y neighbour), values from the
// tables: fb0 = (f0_p + f0_q)/2, fb1 = (f1_p + f1_q)/2, gL = (L_q - L_p)/ds,
// gU = (u_q - u_p)/ds.
//
// D: the face flux F = fb0 gL + fb1 gU enters D_p with +1/ds and D_q with
// -1/ds, so its cotangent weight is mu = (lambda_p - lambda_q)/ds and
//   dF/du_p = f0'_p gL/2 + f1'_p gU/2 - fb1/ds,  dF/du_q = f0'_q gL/2 + f1'_q gU/2 + fb1/ds,
//   dF/dL_q = -dF/dL_p = fb0/ds,                 dF/dkappa = fb1 gU / kappa.
//
// A line row (I + theta dt J) w: the face's part of rows p (+) and q (-),
// times theta dt/ds, is
//   Phi = fb0 W3 + gL (f0'_p w_p + f0'_q w_q)/2 + gU (f1'_p w_p + f1'_q w_q)/2 + fb1 (w_q - w_p)/ds,
// W3 = sum over columns p-1..p+2 of the along-line third difference of w
// (a constant), so with mu = theta dt (lambda_p - lambda_q)/ds
//   dPhi/du_p = f0'_p W3/2 + gL f0''_p w_p/2 + gU f1''_p w_p/2 + f1'_p (w_q - w_p)/(2 ds)
//               - (f1'_p w_p + f1'_q w_q)/(2 ds),
//   dPhi/du_q = f0'_q W3/2 + gL f0''_q w_q/2 + gU f1''_q w_q/2 + f1'_q (w_q - w_p)/(2 ds)
//               + (f1'_p w_p + f1'_q w_q)/(2 ds),
//   dPhi/dL_q = -dPhi/dL_p = (f0'_p w_p + f0'_q w_q)/(2 ds),
//   dPhi/dkappa = [gU (f1'_p w_p + f1'_q w_q)/2 + fb1 (w_q - w_p)/ds] / kappa.
//
// Pass 1 (one thread per cell j, over the faces that touch j): the direct
// u_j terms go to ubar_j, the L_j terms to Lbar_j, and the kappa terms of
// the faces whose p is j to a per-block sum.  Pass 2: ubar_j += the
// transposed five-point Laplacian of Lbar (symmetric, with reflection).

struct FaceVals {
  double up, uq, f0p, f0q, f1p, f1q, d0p, d0q, d1p, d1q, e0p, e0q, e1p, e1q, gL, gU;
};

__device__ __forceinline__ FaceVals face_vals(const AdjK& M, const double* __restrict__ u, const Tables& T,
                                              size_t p, size_t q) {
  FaceVals v;
  v.up = u[p];
  v.uq = u[q];
  v.f0p = T.f0[p];
  v.f0q = T.f0[q];
  v.f1p = T.f1[p];
  v.f1q = T.f1[q];
  v.d0p = T.d0[p];
  v.d0q = T.d0[q];
  v.d1p = T.d1[p];
  v.d1q = T.d1[q];
  v.e0p = T.e0[p];
  v.e0q = T.e0[q];
  v.e1p = T.e1[p];
  v.e1q = T.e1[q];
  v.gL = (T.lap[q] - T.lap[p]) * M.inv_ds;
  v.gU = (v.uq - v.up) * M.inv_ds;
  return v;
}

constexpr int kVjpThreads = 128;

__device__ __forceinline__ void block_sum_to(double v, double* __restrict__ part) {
  __shared__ double s[kVjpThreads];
  s[threadIdx.x] = v;
  __syncthreads();
  for (int h = kVjpThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s[0];
}

// D: ubar_j += scale (D'^T lambda)_j (direct part), Lbar_j = its L_j part,
// part[block] = scale lambda^T dD/dkappa over the block's cells.
__global__ void __launch_bounds__(kVjpThreads) k_vjp_D(AdjK M, const double* __restrict__ u, Tables T,
                                                        const double* __restrict__ lam, double scale,
                                                        double* __restrict__ ubar, double* __restrict__ Lbar,
                                                        double* __restrict__ part) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  double du = 0.0, dL = 0.0, dk = 0.0;
  if (i < M.nx) {
    const size_t c = (size_t)j * M.nx + i;
    const double inv_kappa = M.model == TF_MODEL_LINEAR ? 0.0 : 1.0 / M.kappa;
    // faces (c-dir, c) with c as q and (c, c+dir) with c as p, dir = x, y
    for (int dir = 0; dir < 2; ++dir) {
      const bool has_lo = dir == 0 ? i > 0 : j > 0;
      const bool has_hi = dir == 0 ? i + 1 < M.nx : j + 1 < M.ny;
      const size_t step = dir == 0 ? 1 : (size_t)M.nx;
      for (int side = 0; side < 2; ++side) {
        if (side == 0 ? !has_lo : !has_hi) continue;
        const size_t p = side == 0 ? c - step : c, q = p + step;
        const FaceVals v = face_vals(M, u, T, p, q);
        const double fb0 = 0.5 * (v.f0p + v.f0q), fb1 = 0.5 * (v.f1p + v.f1q);
        const double mu = scale * (lam[p] - lam[q]) * M.inv_ds;
        if (side == 0) {  // c is q
          du += mu * (0.5 * v.d0q * v.gL + 0.5 * v.d1q * v.gU + fb1 * M.inv_ds);
          dL += mu * fb0 * M.inv_ds;
        } else {  // c is p
          du += mu * (0.5 * v.d0p * v.gL + 0.5 * v.d1p * v.gU - fb1 * M.inv_ds);
          dL -= mu * fb0 * M.inv_ds;
          dk += mu * fb1 * v.gU * inv_kappa;
        }
      }
    }
    ubar[c] += du;
    Lbar[c] = dL;
  }
  block_sum_to(dk, part);
}

// A line row along DIR: ubar_j += scale ([d_u (A(u) w)]^T lambda)_j (direct
// part), Lbar_j = its L_j part, part[block] = scale lambda^T d(A w)/dkappa.
template <int DIR>
__global__ void __launch_bounds__(kVjpThreads) k_vjp_line(AdjK M, const double* __restrict__ u, Tables T,
                                                           const double* __restrict__ w,
                                                           const double* __restrict__ lam, double scale,
                                                           double* __restrict__ ubar, double* __restrict__ Lbar,
                                                           double* __restrict__ part) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  double du = 0.0, dL = 0.0, dk = 0.0;
  if (i < M.nx) {
    const size_t c = (size_t)j * M.nx + i;
    const int n = DIR == 0 ? M.nx : M.ny, t = DIR == 0 ? i : j;
    const size_t step = DIR == 0 ? 1 : (size_t)M.nx;
    const double inv_kappa = M.model == TF_MODEL_LINEAR ? 0.0 : 1.0 / M.kappa;
    const double ids3 = M.inv_ds * M.inv_ds * M.inv_ds;
    for (int side = 0; side < 2; ++side) {
      const int pt = side == 0 ? t - 1 : t, qt = pt + 1;  // line indices of p, q
      if (pt < 0 || qt >= n) continue;
      const size_t p = c - (size_t)(t - pt) * step, q = p + step;
      const FaceVals v = face_vals(M, u, T, p, q);
      const double wp = w[p], wq = w[q];
      // W3: the along-line third difference of w over columns p-1..p+2
      double W3 = 0.0;
      for (int a = 0; a < 4; ++a) {
        const int col = pt - 1 + a;
        if (col < 0 || col >= n) continue;
        const double dl = (dlap_line(qt, col, n) - dlap_line(pt, col, n)) * ids3;
        W3 += dl * w[(size_t)((long long)c + (long long)(col - t) * (long long)step)];
      }
      const double fb1 = 0.5 * (v.f1p + v.f1q);
      const double s0 = v.d0p * wp + v.d0q * wq, s1 = v.d1p * wp + v.d1q * wq;
      const double mu = scale * M.tdt * (lam[p] - lam[q]) * M.inv_ds;
      if (side == 0) {  // c is q
        du += mu * (0.5 * v.d0q * W3 + 0.5 * v.gL * v.e0q * wq + 0.5 * v.gU * v.e1q * wq +
                    0.5 * v.d1q * (wq - wp) * M.inv_ds + 0.5 * s1 * M.inv_ds);
        dL += mu * 0.5 * s0 * M.inv_ds;
      } else {  // c is p
        du += mu * (0.5 * v.d0p * W3 + 0.5 * v.gL * v.e0p * wp + 0.5 * v.gU * v.e1p * wp +
                    0.5 * v.d1p * (wq - wp) * M.inv_ds - 0.5 * s1 * M.inv_ds);
        dL -= mu * 0.5 * s0 * M.inv_ds;
        dk += mu * (0.5 * v.gU * s1 + fb1 * (wq - wp) * M.inv_ds) * inv_kappa;
      }
    }
    ubar[c] += du;
    Lbar[c] = dL;
  }
  block_sum_to(dk, part);
}

// ubar_j += (sum over neighbours k of Lbar_k - (neighbours) Lbar_j) / ds^2:
// the transpose of the five-point Laplacian with reflection.
__global__ void k_lap_t(AdjK M, const double* __restrict__ Lbar, double* __restrict__ ubar) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= M.nx) return;
  const size_t c = (size_t)j * M.nx + i;
  const double lc = Lbar[c];
  double s = 0.0;
  if (i + 1 < M.nx) s += Lbar[c + 1] - lc;
  if (i > 0) s += Lbar[c - 1] - lc;
  if (j + 1 < M.ny) s += Lbar[c + M.nx] - lc;
  if (j > 0) s += Lbar[c - M.nx] - lc;
  ubar[c] += s * M.inv_ds * M.inv_ds;
}

// Band of A along DIR at every cell: band[d * N + c] (values only).
template <int DIR>
__global__ void k_band(AdjK M, const double* __restrict__ u, Tables T, double* __restrict__ band) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= M.nx) return;
  double b[5];
  row_band<DIR>(M, u, T, i, j, b);
  const size_t N = (size_t)M.nx * M.ny, c = (size_t)j * M.nx + i;
  for (int d = 0; d < 5; ++d) band[d * N + c] = b[d];
}

// Transposed pentadiagonal solves A^T x = r along every line of direction
// DIR, elimination without pivoting (bandwidth 2), two threads per line
// (lanes 2j, 2j+1 of the block): a twisted elimination.  Row t of A^T holds
// A[t+d-2][t] = band[4-d] of row t+d-2.
//  - The top thread eliminates the lower entries with pivots 0 .. m-1, in
//    the line's order; the bottom thread eliminates the upper entries with
//    pivots n-1 .. m+2, in reversed order (the same code on the reversed
//    line, bands mirrored).  Both leave rows m, m+1 updated in their window.
//  - Each side's multipliers read only entries the other side never
//    changes, so the two updates of rows m, m+1 add: the 2 x 2 system for
//    x_m, x_{m+1} is the original block plus both sides' changes.
//  - The top thread solves it and both substitute back, outwards.
// Lines shorter than 8 are not split.  scratch: 4 values per cell (the
// eliminated row and right side).
constexpr int kSolveLines = 4;  // lines per block, two threads each

template <int DIR>
__global__ void __launch_bounds__(2 * kSolveLines) k_solve_t(int nx, int ny, const double* __restrict__ band,
                                                            const double* __restrict__ r, double* __restrict__ x,
                                                            double* __restrict__ scratch) {
  const int half = threadIdx.x & 1;
  const int line = blockIdx.x * kSolveLines + (threadIdx.x >> 1);
  const int nlines = DIR == 0 ? ny : nx, n = DIR == 0 ? nx : ny;
  const bool active = line < nlines;  // inactive threads still join the shuffles
  const unsigned pair = 3u << (threadIdx.x & ~1);
  const size_t N = (size_t)nx * ny;
  const int m = n >= 8 ? n / 2 : n;  // top pivots 0 .. m-1
  const bool twisted = m < n;
  // pivots and rows (pivots plus the two seam rows) of this thread, in its
  // own orientation: position p is row p (top) or n-1-p (bottom)
  const int npiv = !active ? 0 : half == 0 ? m : (twisted ? n - m - 2 : 0);
  const int nrows = !active ? 0 : (half == 0 ? (twisted ? m + 2 : n) : (twisted ? n - m : 0));
  auto row_of = [&](int p) -> int { return half == 0 ? p : n - 1 - p; };
  auto idx = [&](int t) -> size_t { return DIR == 0 ? (size_t)line * nx + t : (size_t)t * nx + line; };
  auto B = [&](int row, int d) -> double { return (row < 0 || row >= n) ? 0.0 : band[d * N + idx(row)]; };
  // transposed row at position p, oriented: (lo2, lo1, dg, up1, up2)
  auto trow = [&](int p, double& lo2, double& lo1, double& dg, double& up1, double& up2) {
    const int t = row_of(p);
    const double e0 = B(t - 2, 4), e1 = B(t - 1, 3), e3 = B(t + 1, 1), e4 = B(t + 2, 0);
    dg = B(t, 2);
    lo2 = half == 0 ? e0 : e4;
    lo1 = half == 0 ? e1 : e3;
    up1 = half == 0 ? e3 : e1;
    up2 = half == 0 ? e4 : e0;
  };
  double* sd = scratch;          // reciprocal of the eliminated diagonal
  double* s1 = scratch + N;      // eliminated first super-diagonal (oriented)
  double* s2 = scratch + 2 * N;  // second super-diagonal (oriented)
  double* sy = scratch + 3 * N;  // eliminated right side
  // window: positions k (a*), k+1 (b*), k+2 (c*); positions k+2..k+5 are
  // loaded four steps ahead into a ring (slot = position mod 4) so that the
  // loads overlap the elimination chain
  double a_lo2 = 0.0, a_lo1 = 0.0, a_dg = 1.0, a_u1 = 0.0, a_u2 = 0.0, a_y = 0.0;
  double b_lo2 = 0.0, b_lo1 = 0.0, b_dg = 1.0, b_u1 = 0.0, b_u2 = 0.0, b_y = 0.0;
  double c_lo2 = 0.0, c_lo1 = 0.0, c_dg = 1.0, c_u1 = 0.0, c_u2 = 0.0, c_y = 0.0;
  double p_lo2[4], p_lo1[4], p_dg[4], p_u1[4], p_u2[4], p_y[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    p_lo2[q] = p_lo1[q] = p_u1[q] = p_u2[q] = p_y[q] = 0.0;
    p_dg[q] = 1.0;
  }
  if (nrows > 0) {
    trow(0, a_lo2, a_lo1, a_dg, a_u1, a_u2);
    a_y = r[idx(row_of(0))];
  }
  if (nrows > 1) {
    trow(1, b_lo2, b_lo1, b_dg, b_u1, b_u2);
    b_y = r[idx(row_of(1))];
  }
#pragma unroll
  for (int q = 2; q < 6; ++q) {
    if (q < nrows) {
      trow(q, p_lo2[q & 3], p_lo1[q & 3], p_dg[q & 3], p_u1[q & 3], p_u2[q & 3]);
      p_y[q & 3] = r[idx(row_of(q))];
    }
  }
  for (int k0 = 0; k0 < npiv; k0 += 4) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = k0 + q, sl = (q + 2) & 3;  // ring slot of position k + 2
      if (k < npiv) {
        if (k + 2 < nrows) {
          c_lo2 = p_lo2[sl];
          c_lo1 = p_lo1[sl];
          c_dg = p_dg[sl];
          c_u1 = p_u1[sl];
          c_u2 = p_u2[sl];
          c_y = p_y[sl];
        }
        if (k + 6 < nrows) {
          trow(k + 6, p_lo2[sl], p_lo1[sl], p_dg[sl], p_u1[sl], p_u2[sl]);
          p_y[sl] = r[idx(row_of(k + 6))];
        }
        const double inv = 1.0 / a_dg;
        if (k + 1 < nrows) {
          const double l = b_lo1 * inv;
          b_dg -= l * a_u1;
          b_u1 -= l * a_u2;
          b_y -= l * a_y;
        }
        if (k + 2 < nrows) {
          const double l = c_lo2 * inv;
          c_lo1 -= l * a_u1;
          c_dg -= l * a_u2;
          c_y -= l * a_y;
        }
        const size_t ck = idx(row_of(k));
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
  // the seam: a = the first row after this thread's pivots, b = the second
  // (top: rows m, m+1; bottom: rows m+1, m)
  double x1 = 0.0, x2 = 0.0;  // the two unknowns beyond this thread's pivots, nearest first
  if (twisted) {
    // bottom: its changes to rows m (b) and m+1 (a), in the line's orientation
    double o_lo2, o_lo1, o_dg, o_u1, o_u2;
    double d_m_dg = 0.0, d_m_up = 0.0, d_m_y = 0.0, d_p_lo = 0.0, d_p_dg = 0.0, d_p_y = 0.0;
    if (half == 1 && active) {
      trow(npiv + 1, o_lo2, o_lo1, o_dg, o_u1, o_u2);  // row m, mirrored: lo1 = column m+1
      d_m_dg = b_dg - o_dg;
      d_m_up = b_lo1 - o_lo1;
      d_m_y = b_y - r[idx(m)];
      trow(npiv, o_lo2, o_lo1, o_dg, o_u1, o_u2);  // row m+1, mirrored: up1 = column m
      d_p_dg = a_dg - o_dg;
      d_p_lo = a_u1 - o_u1;
      d_p_y = a_y - r[idx(m + 1)];
    }
    d_m_dg = __shfl_sync(pair, d_m_dg, (threadIdx.x & ~1) + 1);
    d_m_up = __shfl_sync(pair, d_m_up, (threadIdx.x & ~1) + 1);
    d_m_y = __shfl_sync(pair, d_m_y, (threadIdx.x & ~1) + 1);
    d_p_lo = __shfl_sync(pair, d_p_lo, (threadIdx.x & ~1) + 1);
    d_p_dg = __shfl_sync(pair, d_p_dg, (threadIdx.x & ~1) + 1);
    d_p_y = __shfl_sync(pair, d_p_y, (threadIdx.x & ~1) + 1);
    double xm = 0.0, xp = 0.0;
    if (half == 0 && active) {
      // top's window: a = row m (dg, up1 = column m+1), b = row m+1 (lo1 = column m, dg)
      const double S00 = a_dg + d_m_dg, S01 = a_u1 + d_m_up, S10 = b_lo1 + d_p_lo, S11 = b_dg + d_p_dg;
      const double y0 = a_y + d_m_y, y1 = b_y + d_p_y;
      const double idet = 1.0 / (S00 * S11 - S01 * S10);
      xm = (y0 * S11 - S01 * y1) * idet;
      xp = (S00 * y1 - S10 * y0) * idet;
      x[idx(m)] = xm;
    }
    xm = __shfl_sync(pair, xm, threadIdx.x & ~1);
    xp = __shfl_sync(pair, xp, threadIdx.x & ~1);
    if (half == 1 && active) x[idx(m + 1)] = xp;
    x1 = half == 0 ? xm : xp;
    x2 = half == 0 ? xp : xm;
  }
#pragma unroll 4
  for (int k = npiv - 1; k >= 0; --k) {
    const size_t ck = idx(row_of(k));
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

// dkappa/dtheta_c when kappa = (1 - cos theta_c)/(b M) was derived from the
// contact angle (power law), M = (n - m)/((m - 1)(n - 1)): sin theta_c/(b M);
// 0 when kappa was given.
double dkappa_dtheta(const tf_ctx& c) {
  if (c.p.kappa > 0.0 || c.p.model != TF_MODEL_POWERLAW) return 0.0;
  const double Mf = (double)(c.p.n - c.p.m) / ((double)(c.p.m - 1) * (double)(c.p.n - 1));
  return sin(c.p.contact_angle) / (c.p.b * Mf);
}

double g_adj_ms[kGroups];  // last call's group times (the library's callers
                           // serialise adjoint calls per process for timing)

}  // namespace

extern "C" int tf_adjoint_timing(double* ms, int n) {
  if (!ms || n < 1) return TF_ERR_ARG;
  for (int g = 0; g < n && g < kGroups; ++g) ms[g] = g_adj_ms[g];
  return TF_OK;
}

namespace {

// Reverse workspace, kept by the context: band (5), lam_y, lam_x, bbar,
// scratch (4; its first grid is also Lbar), tables (7), the kappa partial
// sums (one per 128-cell block of a row, per derivative launch) and, when
// asked for, room for one step's iterates (u_1..u_K, w_0..w_{K-1},
// v_0..v_{K-1}).
struct RevWork {
  double *band, *lam_y, *lam_x, *bbar, *scratch, *part, *iter;
  Tables Tb;
  int npart, nkl;
};

int rev_workspace(tf_ctx* c, int K, bool iterates, RevWork* w) {
  const size_t N = c->N;
  w->npart = ((c->p.nx + kVjpThreads - 1) / kVjpThreads) * c->p.ny;
  w->nkl = 3 * K + 1;
  const size_t rev = 19 * N + (size_t)w->npart * w->nkl;
  const size_t bytes = (rev + (iterates ? (size_t)3 * K * N : 0)) * sizeof(double);
  if (c->adj_bytes < bytes) {
    if (c->adj_ws) cudaFree(c->adj_ws);
    c->adj_ws = nullptr;
    c->adj_bytes = 0;
    if (cudaMalloc(&c->adj_ws, bytes) != cudaSuccess) {
      cudaGetLastError();
      return TF_ERR_NOMEM;
    }
    c->adj_bytes = bytes;
  }
  double* base = (double*)c->adj_ws;
  w->band = base;
  w->lam_y = base + 5 * N;
  w->lam_x = base + 6 * N;
  w->bbar = base + 7 * N;
  w->scratch = base + 8 * N;
  w->Tb.f0 = base + 12 * N;
  w->Tb.f1 = w->Tb.f0 + N;
  w->Tb.d0 = w->Tb.f1 + N;
  w->Tb.d1 = w->Tb.d0 + N;
  w->Tb.e0 = w->Tb.d1 + N;
  w->Tb.e1 = w->Tb.e0 + N;
  w->Tb.lap = w->Tb.e1 + N;
  w->part = base + 19 * N;
  w->iter = iterates ? base + rev : nullptr;
  return TF_OK;
}

// K iterations of the FP64 path from u^n = U[0], keeping u_1..u_K in
// U[1..K] and w_k, v_k: queued without waiting (the forward step's kernels
// in its order, so its bits).
int adj_forward(tf_ctx* c, double dt, int K, double* const* U, double* const* W, double* const* V) {
  return tf::fixed_iterates(*c, dt, K, U, W, V);
}

// The reverse of one step from its iterates (U[0] = u^n, U[1..K-1], W, V):
// g_h = (du^K/du^n)^T g; *kbar receives the step's kappa cotangent (partial
// sums added on the host in a fixed order).  Runs on T.st and synchronises
// it; reads only the context's parameters and its adjoint workspace, so a
// forward may run on the context's own stream at the same time.
int adj_reverse(tf_ctx* c, const RevWork& R, const double* const* U, const double* const* W,
                const double* const* V, double dt, int K, const double* g, double* g_h, double* kbar,
                GroupTimer& T) {
  const int nx = c->p.nx, ny = c->p.ny;
  const size_t N = c->N;
  cudaStream_t st = T.st;  // the stream the reverse runs on
  const double* h_old = U[0];
  double *band = R.band, *lam_y = R.lam_y, *lam_x = R.lam_x, *bbar = R.bbar, *scratch = R.scratch;
  double* part = R.part;
  double* Lbar = scratch;  // free once a transposed solve has finished
  const Tables& Tb = R.Tb;
  const int npart = R.npart, nkl = R.nkl;
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
  const dim3 gv((nx + kVjpThreads - 1) / kVjpThreads, ny), bv(kVjpThreads);
  // one thread per line, kSolveLines per block: the elimination is a chain of
  // dependent FP64 operations, and a warp's FP64 instruction takes longer the
  // more lanes it carries, so few lines per warp over many SMs run faster
  const int nl_x = (ny + kSolveLines - 1) / kSolveLines, nl_y = (nx + kSolveLines - 1) / kSolveLines;
  const int nb = (int)((N + 255) / 256);
  int kl = 0;  // derivative launches so far (each writes one row of partials)

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
    k_solve_t<1><<<nl_y, 2 * kSolveLines, 0, st>>>(nx, ny, band, g_h, lam_y, scratch);
    T.end(t);
    t = T.begin(kGLineY);
    k_vjp_line<1><<<gv, bv, 0, st>>>(M, uk, Tb, V[k], lam_y, -1.0, g_h, Lbar, part + (size_t)(kl++) * npart);
    k_lap_t<<<g2, b2, 0, st>>>(M, Lbar, g_h);
    T.end(t);
    // w_k = A_x(u_k)^-1 (-G(u_k))
    t = T.begin(kGBand);
    k_band<0><<<g2, b2, 0, st>>>(M, uk, Tb, band);
    T.end(t);
    t = T.begin(kGSolve);
    k_solve_t<0><<<nl_x, 2 * kSolveLines, 0, st>>>(nx, ny, band, lam_y, lam_x, scratch);
    T.end(t);
    t = T.begin(kGLineX);
    k_vjp_line<0><<<gv, bv, 0, st>>>(M, uk, Tb, W[k], lam_x, -1.0, g_h, Lbar, part + (size_t)(kl++) * npart);
    k_lap_t<<<g2, b2, 0, st>>>(M, Lbar, g_h);
    T.end(t);
    // -G(u_k) = -u_k - theta dt D(u_k) + b
    k_axpy<<<nb, 256, 0, st>>>(N, -1.0, lam_x, g_h);
    k_axpy<<<nb, 256, 0, st>>>(N, 1.0, lam_x, bbar);
    t = T.begin(kGD);
    k_vjp_D<<<gv, bv, 0, st>>>(M, uk, Tb, lam_x, -M.tdt, g_h, Lbar, part + (size_t)(kl++) * npart);
    k_lap_t<<<g2, b2, 0, st>>>(M, Lbar, g_h);
    T.end(t);
  }
  // b = u^n - (1-theta) dt D(u^n); the tables hold u_0 = h_old
  const double ex = (1.0 - theta) * dt;
  k_axpy<<<nb, 256, 0, st>>>(N, 1.0, bbar, g_h);
  {
    const int t = T.begin(kGD);
    k_vjp_D<<<gv, bv, 0, st>>>(M, h_old, Tb, bbar, -ex, g_h, Lbar, part + (size_t)(kl++) * npart);
    k_lap_t<<<g2, b2, 0, st>>>(M, Lbar, g_h);
    T.end(t);
  }
  // kappa: the partial sums added on the host in a fixed order
  std::vector<double> hp((size_t)nkl * npart);
  {
    const int t = T.begin(kGKappa);
    const cudaError_t e = cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    T.end(t);
    if (e != cudaSuccess) return TF_ERR_CUDA;
  }
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return TF_ERR_CUDA;
  if (T.err != cudaSuccess) return TF_ERR_CUDA;
  double ks = 0.0;
  for (double v : hp) ks += v;
  *kbar = ks;
  return TF_OK;
}

}  // namespace

extern "C" int tf_adjoint_step(tf_ctx* c, const double* h_old, double dt, int K, const double* g,
                               double* h_new, double* g_h, double* g_kappa, double* g_theta) {
  if (!c || !h_old || !g || !g_h || K < 1 || K > 64 || !(dt > 0.0) || !isfinite(dt)) return TF_ERR_ARG;
  if (c->p.precision != TF_FP64) return TF_ERR_ARG;
  if (c->p.model != TF_MODEL_POWERLAW && c->p.model != TF_MODEL_LINEAR) return TF_ERR_ARG;
  if (g_h == h_old || g_h == g || (h_new && (h_new == h_old || h_new == g_h))) return TF_ERR_ARG;
  const size_t N = c->N;
  RevWork R;
  int r = rev_workspace(c, K, true, &R);
  if (r) return r;
  std::vector<double*> U(K + 1), W(K), V(K);
  U[0] = const_cast<double*>(h_old);
  for (int k = 0; k < K; ++k) {
    U[k + 1] = R.iter + (size_t)k * N;
    W[k] = R.iter + (size_t)(K + k) * N;
    V[k] = R.iter + (size_t)(2 * K + k) * N;
  }
  GroupTimer T;
  T.st = c->stream;
  const int tf0 = T.begin(kGForward);
  r = adj_forward(c, dt, K, U.data(), W.data(), V.data());
  if (r) return r;
  T.end(tf0);
  if (h_new && cudaMemcpyAsync(h_new, U[K], N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
    return TF_ERR_CUDA;
  double kbar = 0.0;
  r = adj_reverse(c, R, U.data(), W.data(), V.data(), dt, K, g, g_h, &kbar, T);
  if (r) return r;
  T.collect(g_adj_ms);
  if (g_kappa) *g_kappa = kbar;
  if (g_theta) *g_theta = kbar * dkappa_dtheta(*c);
  return TF_OK;
}

// ---------------------------------------------------------------------------
// Trajectories: N fixed steps with uniform checkpoints.  The forward keeps
// u^n at n = 0, e, 2e, ...; the reverse takes the segments last to first,
// runs a segment's e steps again from its checkpoint keeping every step's
// iterates (the same bits as the forward: tf_newton_iteration equals the
// fused step), and reverses them, the cotangent ping-ponging between two
// grids.  Both halves are chains of dependent FP64 operations that leave
// most of the GPU idle, so segment s-1 is run again (a host worker thread,
// the context's stream, one bank of iterates) while segment s is reversed
// (this thread, the tape's own stream, the other bank).

struct tf_tape {
  tf_ctx* c;
  int nsteps, K, every, nckpt;
  double dt;
  double* mem;  // nckpt checkpoints, 2 banks of every x 3K iterate grids, 2 cotangents
  size_t bytes;
  cudaStream_t rev;  // the reverse's stream
  bool forward_done;
  double ms[2 + kGroups];
};

namespace {

double* tape_ckpt(tf_tape* t, int s) { return t->mem + (size_t)s * t->c->N; }
// grid q (0 .. 3K-1) of segment step i in bank b: u_1..u_K, w_0..w_{K-1},
// v_0..v_{K-1}
double* tape_iter(tf_tape* t, int b, int i, int q) {
  return t->mem + ((size_t)t->nckpt + ((size_t)b * t->every + i) * 3 * t->K + q) * t->c->N;
}
double* tape_cot(tf_tape* t, int i) {
  return t->mem + ((size_t)t->nckpt + (size_t)2 * t->every * 3 * t->K + i) * t->c->N;
}

// Event-timed region on the context's stream, added to *acc.
struct RegionTimer {
  cudaStream_t st;
  cudaEvent_t a = nullptr, b = nullptr;
  explicit RegionTimer(cudaStream_t s) : st(s) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
  }
  void stop(double* acc) {
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) == cudaSuccess) *acc += ms;
  }
  ~RegionTimer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

}  // namespace

extern "C" int tf_tape_create(tf_ctx* c, int nsteps, int K, double dt, int every, tf_tape** out) {
  if (!out) return TF_ERR_ARG;
  *out = nullptr;
  if (!c || nsteps < 1 || K < 1 || K > 64 || !(dt > 0.0) || !isfinite(dt) || every < 0 || every > nsteps)
    return TF_ERR_ARG;
  if (c->p.precision != TF_FP64) return TF_ERR_ARG;
  if (c->p.model != TF_MODEL_POWERLAW && c->p.model != TF_MODEL_LINEAR) return TF_ERR_ARG;
  if (every == 0) {
    every = (int)ceil(sqrt((double)nsteps));
    while ((long long)(every - 1) * (every - 1) >= nsteps) --every;  // sqrt rounding
    while ((long long)every * every < nsteps) ++every;
  }
  tf_tape* t = (tf_tape*)calloc(1, sizeof(tf_tape));
  if (!t) return TF_ERR_NOMEM;
  t->c = c;
  t->nsteps = nsteps;
  t->K = K;
  t->dt = dt;
  t->every = every;
  t->nckpt = (nsteps + every - 1) / every;
  const size_t grids = (size_t)t->nckpt + (size_t)2 * every * 3 * K + 2;
  t->bytes = grids * c->N * sizeof(double);
  if (cudaMalloc(&t->mem, t->bytes) != cudaSuccess) {
    cudaGetLastError();
    free(t);
    return TF_ERR_NOMEM;
  }
  // the reverse is the longer half of each segment's work: its stream gets
  // the highest priority, and the forward of the next segment fills the
  // SMs it leaves idle
  int prio_lo = 0, prio_hi = 0;
  if (cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess) prio_hi = 0;
  if (cudaStreamCreateWithPriority(&t->rev, cudaStreamNonBlocking, prio_hi) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(t->mem);
    free(t);
    return TF_ERR_CUDA;
  }
  *out = t;
  return TF_OK;
}

extern "C" void tf_tape_destroy(tf_tape* t) {
  if (!t) return;
  cudaStreamDestroy(t->rev);
  cudaFree(t->mem);
  free(t);
}

extern "C" int tf_tape_info(const tf_tape* t, int* every, int* checkpoints, size_t* bytes, int* forward_done) {
  if (!t) return TF_ERR_ARG;
  if (every) *every = t->every;
  if (checkpoints) *checkpoints = t->nckpt;
  if (bytes) *bytes = t->bytes;
  if (forward_done) *forward_done = t->forward_done ? 1 : 0;
  return TF_OK;
}

extern "C" int tf_tape_timing(const tf_tape* t, double* ms, int n) {
  if (!t || !ms || n < 1) return TF_ERR_ARG;
  for (int g = 0; g < n && g < 2 + kGroups; ++g) ms[g] = t->ms[g];
  return TF_OK;
}

extern "C" int tf_tape_forward(tf_tape* t, const double* h0, double* hT) {
  if (!t || !h0 || !hT) return TF_ERR_ARG;
  tf_ctx& c = *t->c;
  const size_t gb = c.N * sizeof(double);
  const char* lo = (const char*)t->mem;
  const char* hi = lo + t->bytes;
  if (((const char*)hT >= lo && (const char*)hT < hi) || ((const char*)h0 >= lo && (const char*)h0 < hi))
    return TF_ERR_ARG;
  t->forward_done = false;
  t->ms[0] = 0.0;
  cudaStream_t st = c.stream;
  RegionTimer R(st);
  // u^n is written straight into its checkpoint when n % e == 0 (u^0 is
  // copied there), else into one of two scratch grids (the cotangent grids,
  // free until the reverse); the last step writes hT.
  double* scr[2] = {tape_cot(t, 0), tape_cot(t, 1)};
  if (cudaMemcpyAsync(tape_ckpt(t, 0), h0, gb, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return TF_ERR_CUDA;
  const double* cur = tape_ckpt(t, 0);
  for (int n = 0; n < t->nsteps; ++n) {
    double* nxt;
    if (n + 1 == t->nsteps)
      nxt = hT;
    else if ((n + 1) % t->every == 0)
      nxt = tape_ckpt(t, (n + 1) / t->every);
    else
      nxt = cur == scr[0] ? scr[1] : scr[0];
    const int r = tf::fixed_step(c, cur, nxt, t->dt, t->K);
    if (r != TF_OK) return r;
    cur = nxt;
  }
  R.stop(&t->ms[0]);
  t->forward_done = true;
  return TF_OK;
}

namespace {

// Pointers to the iterates of segment s (bank s & 1): step i starts from
// u^{n0+i} (the checkpoint, then the previous step's u_K).
struct SegPtrs {
  std::vector<double*> U, W, V;  // (K + 1), K, K per step
  int len;
};

void seg_ptrs(tf_tape* t, int s, SegPtrs* P) {
  const int K = t->K, n0 = s * t->every, b = s & 1;
  P->len = (n0 + t->every < t->nsteps ? n0 + t->every : t->nsteps) - n0;
  P->U.assign((size_t)t->every * (K + 1), nullptr);
  P->W.assign((size_t)t->every * K, nullptr);
  P->V.assign((size_t)t->every * K, nullptr);
  for (int i = 0; i < P->len; ++i) {
    double** Ui = &P->U[(size_t)i * (K + 1)];
    Ui[0] = i == 0 ? tape_ckpt(t, s) : P->U[(size_t)(i - 1) * (K + 1) + K];
    for (int k = 0; k < K; ++k) {
      Ui[k + 1] = tape_iter(t, b, i, k);
      P->W[(size_t)i * K + k] = tape_iter(t, b, i, K + k);
      P->V[(size_t)i * K + k] = tape_iter(t, b, i, 2 * K + k);
    }
  }
}

// Runs segment s again on the context's stream, keeping its iterates.
int seg_forward(tf_tape* t, const SegPtrs& P, double* ms) {
  tf_ctx& c = *t->c;
  const int K = t->K;
  RegionTimer R(c.stream);
  for (int i = 0; i < P.len; ++i) {
    const int r = adj_forward(&c, t->dt, K, &P.U[(size_t)i * (K + 1)], &P.W[(size_t)i * K], &P.V[(size_t)i * K]);
    if (r) return r;
  }
  if (cudaStreamSynchronize(c.stream) != cudaSuccess) return TF_ERR_CUDA;
  R.stop(ms);
  return TF_OK;
}

}  // namespace

extern "C" int tf_tape_backward(tf_tape* t, const double* g, double* g_h0, double* g_kappa, double* g_theta) {
  if (!t || !g || !g_h0 || !t->forward_done) return TF_ERR_ARG;
  tf_ctx& c = *t->c;
  const int K = t->K;
  const size_t gb = c.N * sizeof(double);
  for (int k = 1; k < 2 + kGroups; ++k) t->ms[k] = 0.0;
  RevWork Rw;
  int r = rev_workspace(&c, K, false, &Rw);
  if (r) return r;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TF_ERR_CUDA;
  // the reverse stream starts after everything queued on the context's
  if (cudaStreamSynchronize(c.stream) != cudaSuccess) return TF_ERR_CUDA;
  double* cot[2] = {tape_cot(t, 0), tape_cot(t, 1)};
  if (cudaMemcpyAsync(cot[0], g, gb, cudaMemcpyDeviceToDevice, t->rev) != cudaSuccess) return TF_ERR_CUDA;
  int cc = 0;
  double kbar = 0.0;
  SegPtrs cur, nxt;
  seg_ptrs(t, t->nckpt - 1, &cur);
  r = seg_forward(t, cur, &t->ms[1]);
  if (r) return r;
  for (int s = t->nckpt - 1; s >= 0; --s) {
    // segment s - 1 runs again on a worker thread while s is reversed here
    int rw = TF_OK;
    double ms_w = 0.0;
    std::thread worker;
    bool ahead = false;  // segment s - 1 already queued on the worker
    if (s > 0) {
      seg_ptrs(t, s - 1, &nxt);
      try {
        worker = std::thread([&]() {
          if (cudaSetDevice(dev) != cudaSuccess) {
            rw = TF_ERR_CUDA;
            return;
          }
          rw = seg_forward(t, nxt, &ms_w);
        });
        ahead = true;
      } catch (...) {  // no thread: run the segments one after the other
      }
    }
    int rr = TF_OK;
    for (int i = cur.len - 1; i >= 0 && rr == TF_OK; --i) {
      GroupTimer T;
      T.st = t->rev;
      double gk = 0.0;
      rr = adj_reverse(&c, Rw, &cur.U[(size_t)i * (K + 1)], &cur.W[(size_t)i * K], &cur.V[(size_t)i * K], t->dt,
                       K, cot[cc], cot[cc ^ 1], &gk, T);
      if (rr != TF_OK) break;
      double ms[kGroups];
      T.collect(ms);
      for (int k = 0; k < kGroups; ++k) t->ms[2 + k] += ms[k];
      cc ^= 1;
      kbar += gk;
    }
    if (worker.joinable()) worker.join();
    if (rr) return rr;
    if (s > 0 && !ahead) rw = seg_forward(t, nxt, &ms_w);
    if (rw) return rw;
    t->ms[1] += ms_w;
    std::swap(cur, nxt);
  }
  if (cudaMemcpyAsync(g_h0, cot[cc], gb, cudaMemcpyDeviceToDevice, t->rev) != cudaSuccess ||
      cudaStreamSynchronize(t->rev) != cudaSuccess)
    return TF_ERR_CUDA;
  if (g_kappa) *g_kappa = kbar;
  if (g_theta) *g_theta = kbar * dkappa_dtheta(c);
  return TF_OK;
}
