// tf_sweeps.cuh -- residual kernel and the line machinery shared by the
// sweeps of one Newton--ADI iteration (eqs. JacobianSystem1-3):
//
//   k_rhs     2-D tiles: r = -G(u_k) in HP, stored in LP (the x right side);
//             in FP32-bulk also the FP32 film copy that the sweeps stage
//   (the x and y sweeps that solve the lines are in tf_line_sweeps.cuh)
//
// Each line is solved exactly by a twisted ("meet in the middle") LU
// factorisation without pivoting: one thread eliminates the lower band from
// the first cell down to the middle, a second thread eliminates the upper
// band from the last cell up to the middle, the four unknowns at the seam
// come from a 4x4 solve with partial pivoting, and each thread then
// back-substitutes its half outward.  This is the LU solve of eq.
// LUFactorization split across two threads, so every line keeps two
// threads busy instead of one.  The band of each row is assembled on the
// fly from the staged film tile (Sec. Flux Discretization with the J_x/J_y
// split of eq. DirectionSplit) and never stored; the LU factors of a line
// are stored in global scratch between the forward and the backward pass,
// in layouts where every per-step store and load is a 32-wide coalesced
// access.  Tiles are staged into shared memory with cp.async; wall
// reflection (eq. BoundaryConditions) is folded into the copy addresses.
#pragma once

#include <cuda_pipeline.h>

#include "tf_kernels.cuh"

namespace tf {

// ---------------------------------------------------------------------------
// residual -> right side of the x solve

// Arithmetic of the residual: plain IEEE double, or lazy double-float pairs
// folded (hp_norm) before they are stored in shared memory.
__device__ __forceinline__ double hp_add(double a, double b) { return a + b; }
__device__ __forceinline__ double hp_sub(double a, double b) { return a - b; }
__device__ __forceinline__ double hp_mul(double a, double b) { return a * b; }
__device__ __forceinline__ double hp_norm(double a) { return a; }
__device__ __forceinline__ df64 hp_add(df64 a, df64 b) { return df_add_u(a, b); }
__device__ __forceinline__ df64 hp_sub(df64 a, df64 b) { return df_add_u(a, -b); }
__device__ __forceinline__ df64 hp_mul(df64 a, df64 b) { return df_mul_u(a, b); }
__device__ __forceinline__ df64 hp_norm(df64 a) { return df_norm(a); }

// Film height in HP for the residual (heights are positive and normal;
// anything else fails the step in the y sweep).
template <class HP> __device__ __forceinline__ HP film_hp(double u);
template <> __device__ __forceinline__ double film_hp<double>(double u) { return u; }
template <> __device__ __forceinline__ df64 film_hp<df64>(double u) { return df_of_pos_f64_fast(u); }

template <class HP, int T> struct RhsSmem {
  HP u[T + 4][T + 4];
  HP lap[T + 2][T + 2], f0[T + 2][T + 2], f1[T + 2][T + 2];
  HP fx[T][T + 1], fy[T + 1][T];
};

// KIND kRhsResidual: the residual pass of one Newton iteration.  kRhsExplicit:
// the explicit part b^n = u^n - (1 - theta) dt D(u^n) of a step (eq.
// CrankNicolson), written to bn in HP; rhs, ul and part are unused.
// kRhsBoth: both from one D(u^n) -- b^n, and the residual of the step's
// first iteration (u_0 = u^n) from the stored b^n, as kRhsResidual would
// form it (gscale the explicit part's, gscale2 the residual's).
template <class Mode, int KIND>
__global__ void __launch_bounds__(256, 4)  // shared memory allows 4 blocks per SM: up to 64 registers
    k_rhs(ModelK M, RhsK<typename Mode::HP> RK, const double* __restrict__ u,
          typename Mode::HP* __restrict__ bn,
          typename Mode::LP* __restrict__ rhs, typename Mode::LP* __restrict__ ul,
          PartX* __restrict__ part) {
  typedef typename Mode::HP HP;
  typedef typename Mode::LP LP;
  constexpr int T = 32, NT = 256;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RhsSmem<HP, T>& S = *reinterpret_cast<RhsSmem<HP, T>*>(smem_raw);
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * T, j0 = blockIdx.y * T;
  const MobC<HP>& mc = RK.mc;
  const HP inv_ds2 = RK.inv_ds2;
  for (int k = tid; k < (T + 4) * (T + 4); k += NT) {
    int r = k / (T + 4), c = k - r * (T + 4);
    int gj = reflect_index(j0 - 2 + r, M.ny), gi = reflect_index(x0 - 2 + c, M.nx);
    S.u[r][c] = film_hp<HP>(__ldg(u + (size_t)gj * M.nx + gi));
  }
  __syncthreads();
  const HP four = RK.four;
  for (int k = tid; k < (T + 2) * (T + 2); k += NT) {
    int r = k / (T + 2), c = k - r * (T + 2);
    HP uc = S.u[r + 1][c + 1];
    // lap = (sum of the four neighbours - 4 u) / ds^2; a wall neighbour is
    // the cell itself (reflected tile) and cancels one of the four.
    HP nb = hp_add(hp_add(S.u[r + 1][c + 2], S.u[r + 1][c]), hp_add(S.u[r + 2][c + 1], S.u[r][c + 1]));
    S.lap[r][c] = hp_norm(hp_mul(hp_sub(nb, hp_mul(four, uc)), inv_ds2));
    HP s = rcp(uc), f0, f1;
    mobility(mc, uc, s, f0, f1);
    S.f0[r][c] = hp_norm(f0);
    S.f1[r][c] = hp_norm(f1);
  }
  __syncthreads();
  for (int k = tid; k < T * (T + 1); k += NT) {
    int r = k / (T + 1), c = k - r * (T + 1);
    int gp = x0 - 1 + c;
    HP F = zero<HP>();
    if (gp >= 0 && gp + 1 < M.nx) {
      int rr = r + 1;
      F = hp_norm(hp_add(
          hp_mul(hp_add(S.f0[rr][c], S.f0[rr][c + 1]), hp_sub(S.lap[rr][c + 1], S.lap[rr][c])),
          hp_mul(hp_add(S.f1[rr][c], S.f1[rr][c + 1]), hp_sub(S.u[rr + 1][c + 2], S.u[rr + 1][c + 1]))));
    }
    S.fx[r][c] = F;
  }
  for (int k = tid; k < (T + 1) * T; k += NT) {
    int r = k / T, c = k - r * T;
    int gp = j0 - 1 + r;
    HP F = zero<HP>();
    if (gp >= 0 && gp + 1 < M.ny) {
      int cc = c + 1;
      F = hp_norm(hp_add(
          hp_mul(hp_add(S.f0[r][cc], S.f0[r + 1][cc]), hp_sub(S.lap[r + 1][cc], S.lap[r][cc])),
          hp_mul(hp_add(S.f1[r][cc], S.f1[r + 1][cc]), hp_sub(S.u[r + 2][cc + 1], S.u[r + 1][cc + 1]))));
    }
    S.fy[r][c] = F;
  }
  __syncthreads();
  const HP gscale = RK.gscale;
  LP g = LP(0);  // max |G| in LP: a norm for reporting, not a decision
  for (int k = tid; k < T * T; k += NT) {
    int r = k / T, c = k - r * T;
    int gj = j0 + r, gi = x0 + c;
    if (gj < M.ny && gi < M.nx) {
      const size_t idx = (size_t)gj * M.nx + gi;
      HP dp = hp_add(hp_sub(S.fx[r][c + 1], S.fx[r][c]), hp_sub(S.fy[r + 1][c], S.fy[r][c]));
      if constexpr (KIND == kRhsExplicit) {  // gscale holds (1 - theta) dt / (2 ds^2)
        bn[idx] = hp_norm(hp_sub(S.u[r + 2][c + 2], hp_mul(gscale, dp)));
        continue;
      }
      HP Gv;
      if constexpr (KIND == kRhsBoth) {
        const HP b = hp_norm(hp_sub(S.u[r + 2][c + 2], hp_mul(gscale, dp)));
        bn[idx] = b;
        Gv = hp_norm(hp_add(hp_sub(S.u[r + 2][c + 2], b), hp_mul(RK.gscale2, dp)));
      } else {
        Gv = hp_norm(hp_add(hp_sub(S.u[r + 2][c + 2], bn[idx]), hp_mul(gscale, dp)));
      }
      LP gl = to_lp<LP, HP>(Gv);
      rhs[idx] = -gl;
      // FP32 film for the sweeps: the leading float of the double-float
      // height (the truncated height the FP32 Jacobian is built from)
      if constexpr (sizeof(LP) == 4) ul[idx] = S.u[r + 2][c + 2].hi;
      LP ag = fabs(gl);
      if (!(ag <= g)) g = ag;
    }
  }
  if constexpr (KIND == kRhsExplicit) return;
  for (int o = 16; o > 0; o >>= 1) {
    LP g2 = __shfl_xor_sync(0xffffffffu, g, o);
    if (!(g2 <= g)) g = g2;
  }
  __shared__ LP red[NT / 32];
  if ((tid & 31) == 0) red[tid >> 5] = g;
  __syncthreads();
  if (tid == 0) {
    LP mx = red[0];
    for (int k = 1; k < NT / 32; ++k)
      if (!(red[k] <= mx)) mx = red[k];
    PartX p;
    p.gnorm = (double)mx;
    p.pivot = 0;
    p.pad = 0;
    part[blockIdx.y * gridDim.x + blockIdx.x] = p;
  }
}

// ---------------------------------------------------------------------------
// shared line machinery

// 4x4 solve with partial pivoting (the seam of the twisted factorisation).
template <class LP> __device__ __forceinline__ bool solve4(LP A[4][4], LP b[4], LP x[4]) {
  for (int k = 0; k < 4; ++k) {
    int p = k;
    LP best = fabs(A[k][k]);
    for (int r = k + 1; r < 4; ++r)
      if (fabs(A[r][k]) > best) {
        best = fabs(A[r][k]);
        p = r;
      }
    if (!(best > LP(0)) || !isfinite(best)) return false;
    if (p != k) {
      for (int c = 0; c < 4; ++c) {
        LP t = A[k][c];
        A[k][c] = A[p][c];
        A[p][c] = t;
      }
      LP t = b[k];
      b[k] = b[p];
      b[p] = t;
    }
    LP inv = LP(1) / A[k][k];
    for (int r = k + 1; r < 4; ++r) {
      LP l = A[r][k] * inv;
      for (int c = k; c < 4; ++c) A[r][c] -= l * A[k][c];
      b[r] -= l * b[k];
    }
  }
  for (int k = 3; k >= 0; --k) {
    LP s = b[k];
    for (int c = k + 1; c < 4; ++c) s -= A[k][c] * x[c];
    x[k] = s / A[k][k];
  }
  return true;
}

// Seam: rows m-2, m-1 from the forward (top-down) state S, rows m, m+1 from
// the reversed (bottom-up) state R.  Unknowns (x_{m-2}, x_{m-1}, x_m, x_{m+1}).
template <class LP>
__device__ __forceinline__ bool seam(const LUState<LP>& S, const LUState<LP>& R, LP x[4]) {
  LP A[4][4] = {{LP(1), S.g2, S.d2, LP(0)},
                {LP(0), LP(1), S.g1, S.d1},
                {R.d1, R.g1, LP(1), LP(0)},
                {LP(0), R.d2, R.g2, LP(1)}};
  LP b[4] = {S.z2, S.z1, R.z1, R.z2};
  return solve4(A, b, x);
}

// Where each line splits: the first half covers cells [0, m) with m a
// multiple of the chunk length C near n/2; twisting needs m >= 2 and
// n - m >= 2.
template <int C> __host__ __device__ __forceinline__ int split_point(int n) {
  const int nch = (n + C - 1) / C;
  const int m = ((nch + 1) / 2) * C;
  if (m >= n - 1 || m < 2) return n;  // no second half
  return m;
}

// Per-cell values for the band, read from an LP tile.  U(dr, dc) gives the
// film at an offset from the cell; the tiles hold wall-reflected values, so
// a missing neighbour equals the cell and adds nothing to the Laplacian.
template <class LP, class Acc>
__device__ __forceinline__ CellLP<LP> cell_values(const MobC<LP>& ml, LP inv_ds2, Acc U) {
  CellLP<LP> X;
  LP uc = U(0, 0);
  X.u = uc;
  X.lap = (((U(0, 1) - uc) + (U(0, -1) - uc)) + ((U(1, 0) - uc) + (U(-1, 0) - uc))) * inv_ds2;
  LP s = rcp(uc);
  mobility_all(ml, uc, s, X.f0, X.f1, X.d0, X.d1);
  return X;
}

__device__ __forceinline__ void cp8(void* dst, const void* src) { __pipeline_memcpy_async(dst, src, 8); }
__device__ __forceinline__ void cp4(void* dst, const void* src) { __pipeline_memcpy_async(dst, src, 4); }
template <class T> __device__ __forceinline__ void cpT(T* dst, const T* src) {
  __pipeline_memcpy_async(dst, src, sizeof(T));
}

}  // namespace tf
