// tf_sweeps.cuh -- residual and line-sweep kernels of one Newton--ADI
// iteration (eqs. JacobianSystem1-3):
//
//   k_rhs     2-D tiles: r = -G(u_k) in HP, stored in LP (the x right side)
//   k_xsweep  (I + theta dt J_x) w = r on every row
//   k_ysweep  (I + theta dt J_y) v = w on every column, u_{k+1} = u_k + v,
//             and the block reductions of eq. NewtonError and the norms
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
// are stored in global scratch between the two sweeps, in layouts where
// every per-step store and load is a 32-wide coalesced access.
// Tiles are staged into shared memory with cp.async double buffering; wall
// reflection (eq. BoundaryConditions) is folded into the copy addresses.
#pragma once

#include <cuda_pipeline.h>

#include "tf_kernels.cuh"

namespace tf {

constexpr int kLane = 32;   // lines per block (one warp per half)
constexpr int kChunk = 32;  // cells per staged chunk along a line

// ---------------------------------------------------------------------------
// residual -> right side of the x solve

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

template <class Mode>
__global__ void __launch_bounds__(256)
    k_rhs(ModelK M, StepK K, const double* __restrict__ u, const typename Mode::HP* __restrict__ bn,
          typename Mode::LP* __restrict__ rhs, PartX* __restrict__ part) {
  typedef typename Mode::HP HP;
  typedef typename Mode::LP LP;
  constexpr int T = 32, NT = 256;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RhsSmem<HP, T>& S = *reinterpret_cast<RhsSmem<HP, T>*>(smem_raw);
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * T, j0 = blockIdx.y * T;
  const MobC<HP> mc = mob_consts<HP>(M);
  const HP inv_ds2 = from_f64<HP>(M.inv_ds2);
  for (int k = tid; k < (T + 4) * (T + 4); k += NT) {
    int r = k / (T + 4), c = k - r * (T + 4);
    int gj = reflect_index(j0 - 2 + r, M.ny), gi = reflect_index(x0 - 2 + c, M.nx);
    S.u[r][c] = film_hp<HP>(__ldg(u + (size_t)gj * M.nx + gi));
  }
  __syncthreads();
  for (int k = tid; k < (T + 2) * (T + 2); k += NT) {
    int r = k / (T + 2), c = k - r * (T + 2);
    HP uc = S.u[r + 1][c + 1];
    HP d = ((S.u[r + 1][c + 2] - uc) + (S.u[r + 1][c] - uc)) +
           ((S.u[r + 2][c + 1] - uc) + (S.u[r][c + 1] - uc));
    S.lap[r][c] = d * inv_ds2;
    HP s = rcp(uc), f0, f1;
    mobility(mc, uc, s, f0, f1);
    S.f0[r][c] = f0;
    S.f1[r][c] = f1;
  }
  __syncthreads();
  for (int k = tid; k < T * (T + 1); k += NT) {
    int r = k / (T + 1), c = k - r * (T + 1);
    int gp = x0 - 1 + c;
    HP F = zero<HP>();
    if (gp >= 0 && gp + 1 < M.nx) {
      int rr = r + 1;
      F = (S.f0[rr][c] + S.f0[rr][c + 1]) * (S.lap[rr][c + 1] - S.lap[rr][c]) +
          (S.f1[rr][c] + S.f1[rr][c + 1]) * (S.u[rr + 1][c + 2] - S.u[rr + 1][c + 1]);
    }
    S.fx[r][c] = F;
  }
  for (int k = tid; k < (T + 1) * T; k += NT) {
    int r = k / T, c = k - r * T;
    int gp = j0 - 1 + r;
    HP F = zero<HP>();
    if (gp >= 0 && gp + 1 < M.ny) {
      int cc = c + 1;
      F = (S.f0[r][cc] + S.f0[r + 1][cc]) * (S.lap[r + 1][cc] - S.lap[r][cc]) +
          (S.f1[r][cc] + S.f1[r + 1][cc]) * (S.u[r + 2][cc + 1] - S.u[r + 1][cc + 1]);
    }
    S.fy[r][c] = F;
  }
  __syncthreads();
  const HP gscale = from_f64<HP>(0.5 * M.inv_ds2 * K.theta_dt);
  LP g = LP(0);  // max |G| in LP: a norm for reporting, not a decision
  for (int k = tid; k < T * T; k += NT) {
    int r = k / T, c = k - r * T;
    int gj = j0 + r, gi = x0 + c;
    if (gj < M.ny && gi < M.nx) {
      const size_t idx = (size_t)gj * M.nx + gi;
      HP dp = (S.fx[r][c + 1] - S.fx[r][c]) + (S.fy[r + 1][c] - S.fy[r][c]);
      HP Gv = (S.u[r + 2][c + 2] - bn[idx]) + gscale * dp;
      LP gl = to_lp<LP, HP>(Gv);
      rhs[idx] = -gl;
      LP ag = fabs(gl);
      if (!(ag <= g)) g = ag;
    }
  }
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

// Where each line splits: the first half covers cells [0, m); twisting
// needs m >= 2 and n - m >= 2.
__host__ __device__ __forceinline__ int split_point(int n) {
  int nch = (n + kChunk - 1) / kChunk;
  int m = ((nch + 1) / 2) * kChunk;
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
  mobility(ml, uc, s, X.f0, X.f1);
  mobility_d(ml, uc, s, X.d0, X.d1);
  return X;
}

__device__ __forceinline__ void cp8(void* dst, const void* src) { __pipeline_memcpy_async(dst, src, 8); }
__device__ __forceinline__ void cp4(void* dst, const void* src) { __pipeline_memcpy_async(dst, src, 4); }
template <class T> __device__ __forceinline__ void cpT(T* dst, const T* src) {
  __pipeline_memcpy_async(dst, src, sizeof(T));
}

// ---------------------------------------------------------------------------
// x sweep: block = 32 rows, warp 0 the left halves, warp 1 the right halves.
// Forward stages: film rows j0-1..j0+32 x cols c0-2..c0+33 (FP64, staged then
// converted to LP) and the right side rows j0..j0+31 x cols c0..c0+31.
// Factor scratch (per block of 32 rows): fac[((blk*3 + f)*nx + col)*32 + row].

template <class LP> struct XSweepWarp {
  union {
    struct {
      double u[2][34][36];
      LP r[2][32][kChunk + 1];
    } fw;
    struct {
      LP f[2][3][kChunk][32];
    } bw;
  } st;
  LP ulp[34][37];
  LP wst[32][kChunk + 1];
};
template <class LP> struct XSweepSmem {
  XSweepWarp<LP> w[2];
  LUState<LP> seamS[32], seamR[32];
  LP xs[32][4];
  int ok[32];
};

template <class Mode>
__global__ void __launch_bounds__(64)
    k_xsweep(ModelK M, StepK K, const double* __restrict__ u, typename Mode::LP* __restrict__ rw,
             typename Mode::LP* __restrict__ fac, PartX* __restrict__ part) {
  typedef typename Mode::LP LP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  XSweepSmem<LP>& S = *reinterpret_cast<XSweepSmem<LP>*>(smem_raw);
  const int lane = threadIdx.x & 31, half = threadIdx.x >> 5;
  XSweepWarp<LP>& W = S.w[half];
  const int nx = M.nx, ny = M.ny;
  const int j0 = blockIdx.x * 32;
  const int row = j0 + lane;
  const bool active = row < ny;
  const int m = split_point(nx);
  const bool twisted = m < nx;
  const MobC<LP> ml = mob_consts<LP>(M);
  const LP inv_ds = (LP)M.inv_ds, inv_ds2 = (LP)M.inv_ds2, inv_ds3 = (LP)M.inv_ds3;
  const LP sc = (LP)(K.theta_dt * M.inv_ds);
  LP* facb = fac + (size_t)blockIdx.x * 3 * nx * 32;
  // chunk list of this half: half 0 covers [0, m) left to right; half 1
  // covers [m, nx) right to left, chunks aligned to the right end.
  const int lo = half == 0 ? 0 : m, hi = half == 0 ? m : nx;
  const int nch = half == 0 ? (m + kChunk - 1) / kChunk : (hi - lo + kChunk - 1) / kChunk;
  auto chunk_c0 = [&](int q) {  // first column of chunk q of this half
    return half == 0 ? q * kChunk : max(lo, hi - (q + 1) * kChunk);
  };
  auto chunk_c1 = [&](int q) { return half == 0 ? min(hi, (q + 1) * kChunk) : hi - q * kChunk; };
  int pivot_bad = 0;
  const bool work = half == 0 || twisted;

  auto issue_fw = [&](int q, int buf) {
    const int c0 = chunk_c0(q);
    for (int k = lane; k < 34 * 36; k += 32) {
      int r = k / 36, c = k - r * 36;
      int gj = reflect_index(j0 - 1 + r, ny), gi = reflect_index(c0 - 2 + c, nx);
      cp8(&W.st.fw.u[buf][r][c], u + (size_t)gj * nx + gi);
    }
    const int c1 = chunk_c1(q);
    for (int k = lane; k < 32 * kChunk; k += 32) {
      int r = k / kChunk, c = k - r * kChunk;
      int gj = j0 + r, gi = c0 + c;
      if (gj < ny && gi < c1) cpT(&W.st.fw.r[buf][r][c], rw + (size_t)gj * nx + gi);
    }
    __pipeline_commit();
  };

  LUState<LP> lu;
  lu.reset();
  LP Lf[4] = {LP(0), LP(0), LP(0), LP(0)};
  CellLP<LP> P;
  if (work && nch > 0) {
    issue_fw(0, 0);
    for (int q = 0; q < nch; ++q) {
      const int buf = q & 1;
      if (q + 1 < nch) {
        issue_fw(q + 1, buf ^ 1);
        __pipeline_wait_prior(1);
      } else {
        __pipeline_wait_prior(0);
      }
      __syncwarp();
      for (int k = lane; k < 34 * 36; k += 32) {
        int r = k / 36, c = k - r * 36;
        W.ulp[r][c] = from_f64<LP>(W.st.fw.u[buf][r][c]);
      }
      __syncwarp();
      const int c0 = chunk_c0(q), c1 = chunk_c1(q);
      if (active) {
        // cell (row, col) sits at ulp[lane + 1][col - c0 + 2]
        auto cell = [&](int col) {
          int rr = lane + 1, cc = col - c0 + 2;
          return cell_values<LP>(ml, inv_ds2, [&](int dr, int dc) { return W.ulp[rr + dr][cc + dc]; });
        };
        LP* fg = facb + (size_t)0 * nx * 32;
        LP* fd = facb + (size_t)1 * nx * 32;
        LP* fz = facb + (size_t)2 * nx * 32;
        if (half == 0) {
          if (q == 0) P = cell(0);
          for (int i = c0; i < c1; ++i) {
            LP Rf[4] = {LP(0), LP(0), LP(0), LP(0)};
            CellLP<LP> Q;
            if (i + 1 < nx) {
              Q = cell(i + 1);
              face_dF(P, Q, i > 0, i + 2 < nx, inv_ds, inv_ds3, sc, Rf);
            }
            LP a, b, c, d, e, g, dl, z;
            band_row(Lf, Rf, a, b, c, d, e);
            if (!lu.step(a, b, c, d, e, W.st.fw.r[buf][lane][i - c0], g, dl, z)) pivot_bad = 1;
            fg[(size_t)i * 32 + lane] = g;
            fd[(size_t)i * 32 + lane] = dl;
            fz[(size_t)i * 32 + lane] = z;
            for (int t = 0; t < 4; ++t) Lf[t] = Rf[t];
            P = Q;
          }
        } else {
          if (q == 0) P = cell(nx - 1);
          for (int i = c1 - 1; i >= c0; --i) {
            LP Ff[4] = {LP(0), LP(0), LP(0), LP(0)};  // face (i-1, i)
            CellLP<LP> Q;
            if (i > 0) {
              Q = cell(i - 1);
              face_dF(Q, P, i - 1 > 0, i + 1 < nx, inv_ds, inv_ds3, sc, Ff);
            }
            LP a, b, c, d, e, g, dl, z;
            band_row(Ff, Lf, a, b, c, d, e);  // Lf holds face (i, i+1) here
            if (!lu.step(e, d, c, b, a, W.st.fw.r[buf][lane][i - c0], g, dl, z)) pivot_bad = 1;
            fg[(size_t)i * 32 + lane] = g;
            fd[(size_t)i * 32 + lane] = dl;
            fz[(size_t)i * 32 + lane] = z;
            for (int t = 0; t < 4; ++t) Lf[t] = Ff[t];
            P = Q;
          }
        }
      }
      __syncwarp();
    }
  }
  // seam
  if (half == 0) S.seamS[lane] = lu;
  else S.seamR[lane] = lu;
  __syncthreads();
  if (half == 0 && twisted) {
    LP x[4] = {LP(0), LP(0), LP(0), LP(0)};
    if (!seam(S.seamS[lane], S.seamR[lane], x) && active) pivot_bad = 1;
    for (int t = 0; t < 4; ++t) S.xs[lane][t] = x[t];
  }
  __syncthreads();
  // backward: half 0 walks [0, m) right to left from the seam (or from the
  // end of the line); half 1 walks [m, nx) left to right.  (x1, x2) are the
  // two unknowns solved just before, nearest first; the four seam unknowns
  // x_{m-2..m+1} are taken as known.
  LP x1 = LP(0), x2 = LP(0);
  if (twisted) {
    if (half == 0) {
      x1 = S.xs[lane][2];
      x2 = S.xs[lane][3];
    } else {
      x1 = S.xs[lane][1];
      x2 = S.xs[lane][0];
    }
  }
  auto issue_bw = [&](int q, int buf) {
    const int c0 = chunk_c0(q), c1 = chunk_c1(q);
    for (int f = 0; f < 3; ++f) {
      const LP* src = facb + ((size_t)f * nx + c0) * 32;
      for (int k = lane; k < (c1 - c0) * 32; k += 32) cpT(&W.st.bw.f[buf][f][k >> 5][k & 31], src + k);
    }
    __pipeline_commit();
  };
  if (work && nch > 0) {
    issue_bw(nch - 1, 0);
    int it = 0;
    for (int q = nch - 1; q >= 0; --q, ++it) {
      const int buf = it & 1;
      if (q - 1 >= 0) {
        issue_bw(q - 1, buf ^ 1);
        __pipeline_wait_prior(1);
      } else {
        __pipeline_wait_prior(0);
      }
      __syncwarp();
      const int c0 = chunk_c0(q), c1 = chunk_c1(q);
      if (half == 0) {
        for (int i = c1 - 1; i >= c0; --i) {
          const int k = i - c0;
          LP x = (twisted && i >= m - 2)
                     ? S.xs[lane][i - (m - 2)]
                     : W.st.bw.f[buf][2][k][lane] - W.st.bw.f[buf][0][k][lane] * x1 -
                           W.st.bw.f[buf][1][k][lane] * x2;
          x2 = x1;
          x1 = x;
          W.wst[lane][k] = x;
        }
      } else {
        for (int i = c0; i < c1; ++i) {
          const int k = i - c0;
          LP x = (i <= m + 1) ? S.xs[lane][i - (m - 2)]
                              : W.st.bw.f[buf][2][k][lane] - W.st.bw.f[buf][0][k][lane] * x1 -
                                    W.st.bw.f[buf][1][k][lane] * x2;
          x2 = x1;
          x1 = x;
          W.wst[lane][k] = x;
        }
      }
      __syncwarp();
      for (int k = lane; k < 32 * kChunk; k += 32) {
        int r = k / kChunk, c = k - r * kChunk;
        int gj = j0 + r, gi = c0 + c;
        if (gj < ny && gi < c1) rw[(size_t)gj * nx + gi] = W.wst[r][c];
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // block partial: pivot failures
  __shared__ int s_piv[2];
  int pv = __any_sync(0xffffffffu, pivot_bad);
  if (lane == 0) s_piv[half] = pv;
  __syncthreads();
  if (threadIdx.x == 0) {
    PartX p;
    p.gnorm = 0.0;
    p.pivot = s_piv[0] | s_piv[1];
    p.pad = 0;
    part[blockIdx.x] = p;
  }
}

// ---------------------------------------------------------------------------
// y sweep: block = 32 columns, warp 0 the top halves, warp 1 the bottom
// halves.  Forward stages: film rows r0-2..r0+33 x cols i0-1..i0+32 (FP64,
// converted to LP) and w rows r0..r0+31.  Backward stages: the factors and
// u_k of rows r0..r0+31.  Factor scratch: fac[f*N + row*nx + col].

template <class LP> struct YSweepWarp {
  union {
    struct {
      double u[2][36][34];
      LP w[2][32][32];
    } fw;
    struct {
      LP f[2][3][32][32];
      double u[2][32][32];
    } bw;
  } st;
  LP ulp[36][35];
};
template <class LP> struct YSweepSmem {
  YSweepWarp<LP> w[2];
  LUState<LP> seamS[32], seamR[32];
  LP xs[32][4];
  PartY part[2];
};

template <class Mode>
__global__ void __launch_bounds__(64)
    k_ysweep(ModelK M, StepK K, const double* __restrict__ u, const typename Mode::LP* __restrict__ w,
             typename Mode::LP* __restrict__ fac, double* __restrict__ unew, double* __restrict__ vout,
             PartY* __restrict__ part) {
  typedef typename Mode::LP LP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  YSweepSmem<LP>& S = *reinterpret_cast<YSweepSmem<LP>*>(smem_raw);
  const int lane = threadIdx.x & 31, half = threadIdx.x >> 5;
  YSweepWarp<LP>& W = S.w[half];
  const int nx = M.nx, ny = M.ny;
  const size_t N = (size_t)nx * ny;
  const int i0 = blockIdx.x * 32;
  const int col = i0 + lane;
  const bool active = col < nx;
  const int m = split_point(ny);
  const bool twisted = m < ny;
  const MobC<LP> ml = mob_consts<LP>(M);
  const LP inv_ds = (LP)M.inv_ds, inv_ds2 = (LP)M.inv_ds2, inv_ds3 = (LP)M.inv_ds3;
  const LP sc = (LP)(K.theta_dt * M.inv_ds);
  LP* fg = fac;
  LP* fd = fac + N;
  LP* fz = fac + 2 * N;
  const int lo = half == 0 ? 0 : m, hi = half == 0 ? m : ny;
  const int nch = (hi - lo + kChunk - 1) / kChunk;
  auto chunk_r0 = [&](int q) { return half == 0 ? q * kChunk : max(lo, hi - (q + 1) * kChunk); };
  auto chunk_r1 = [&](int q) { return half == 0 ? min(hi, (q + 1) * kChunk) : hi - q * kChunk; };
  const bool work = half == 0 || twisted;
  int pivot_bad = 0;

  auto issue_fw = [&](int q, int buf) {
    const int r0 = chunk_r0(q), r1 = chunk_r1(q);
    for (int k = lane; k < 36 * 34; k += 32) {
      int r = k / 34, c = k - r * 34;
      int gj = reflect_index(r0 - 2 + r, ny), gi = reflect_index(i0 - 1 + c, nx);
      cp8(&W.st.fw.u[buf][r][c], u + (size_t)gj * nx + gi);
    }
    if (active)
      for (int r = 0; r < r1 - r0; ++r) cpT(&W.st.fw.w[buf][r][lane], w + (size_t)(r0 + r) * nx + col);
    __pipeline_commit();
  };

  LUState<LP> lu;
  lu.reset();
  LP Lf[4] = {LP(0), LP(0), LP(0), LP(0)};
  CellLP<LP> P;
  if (work && nch > 0) {
    issue_fw(0, 0);
    for (int q = 0; q < nch; ++q) {
      const int buf = q & 1;
      if (q + 1 < nch) {
        issue_fw(q + 1, buf ^ 1);
        __pipeline_wait_prior(1);
      } else {
        __pipeline_wait_prior(0);
      }
      __syncwarp();
      for (int k = lane; k < 36 * 34; k += 32) {
        int r = k / 34, c = k - r * 34;
        W.ulp[r][c] = from_f64<LP>(W.st.fw.u[buf][r][c]);
      }
      __syncwarp();
      const int r0 = chunk_r0(q), r1 = chunk_r1(q);
      if (active) {
        auto cell = [&](int row) {  // cell (row, col) sits at ulp[row - r0 + 2][lane + 1]
          int rr = row - r0 + 2, cc = lane + 1;
          return cell_values<LP>(ml, inv_ds2, [&](int dr, int dc) { return W.ulp[rr + dr][cc + dc]; });
        };
        if (half == 0) {
          if (q == 0) P = cell(0);
          for (int i = r0; i < r1; ++i) {
            LP Rf[4] = {LP(0), LP(0), LP(0), LP(0)};
            CellLP<LP> Q;
            if (i + 1 < ny) {
              Q = cell(i + 1);
              face_dF(P, Q, i > 0, i + 2 < ny, inv_ds, inv_ds3, sc, Rf);
            }
            LP a, b, c, d, e, g, dl, z;
            band_row(Lf, Rf, a, b, c, d, e);
            if (!lu.step(a, b, c, d, e, W.st.fw.w[buf][i - r0][lane], g, dl, z)) pivot_bad = 1;
            const size_t idx = (size_t)i * nx + col;
            fg[idx] = g;
            fd[idx] = dl;
            fz[idx] = z;
            for (int t = 0; t < 4; ++t) Lf[t] = Rf[t];
            P = Q;
          }
        } else {
          if (q == 0) P = cell(ny - 1);
          for (int i = r1 - 1; i >= r0; --i) {
            LP Ff[4] = {LP(0), LP(0), LP(0), LP(0)};
            CellLP<LP> Q;
            if (i > 0) {
              Q = cell(i - 1);
              face_dF(Q, P, i - 1 > 0, i + 1 < ny, inv_ds, inv_ds3, sc, Ff);
            }
            LP a, b, c, d, e, g, dl, z;
            band_row(Ff, Lf, a, b, c, d, e);
            if (!lu.step(e, d, c, b, a, W.st.fw.w[buf][i - r0][lane], g, dl, z)) pivot_bad = 1;
            const size_t idx = (size_t)i * nx + col;
            fg[idx] = g;
            fd[idx] = dl;
            fz[idx] = z;
            for (int t = 0; t < 4; ++t) Lf[t] = Ff[t];
            P = Q;
          }
        }
      }
      __syncwarp();
    }
  }
  if (half == 0) S.seamS[lane] = lu;
  else S.seamR[lane] = lu;
  __syncthreads();
  if (half == 0 && twisted) {
    LP x[4] = {LP(0), LP(0), LP(0), LP(0)};
    if (!seam(S.seamS[lane], S.seamR[lane], x) && active) pivot_bad = 1;
    for (int t = 0; t < 4; ++t) S.xs[lane][t] = x[t];
  }
  __syncthreads();
  LP x1 = LP(0), x2 = LP(0);
  if (twisted) {
    if (half == 0) {
      x1 = S.xs[lane][2];
      x2 = S.xs[lane][3];
    } else {
      x1 = S.xs[lane][1];
      x2 = S.xs[lane][0];
    }
  }
  auto issue_bw = [&](int q, int buf) {
    const int r0 = chunk_r0(q), r1 = chunk_r1(q);
    if (active)
      for (int r = 0; r < r1 - r0; ++r) {
        const size_t idx = (size_t)(r0 + r) * nx + col;
        cpT(&W.st.bw.f[buf][0][r][lane], fg + idx);
        cpT(&W.st.bw.f[buf][1][r][lane], fd + idx);
        cpT(&W.st.bw.f[buf][2][r][lane], fz + idx);
        cp8(&W.st.bw.u[buf][r][lane], u + idx);
      }
    __pipeline_commit();
  };
  // Reductions kept off the FP64 pipe in FP32-bulk: the relative update in
  // LP, the minimum as the smallest bit pattern of a positive double (bit
  // patterns of positive doubles order like the values).
  LP err = LP(0);
  unsigned long long hmin_bits = 0x7ff0000000000000ull;  // +inf
  long long mass = 0;
  int nonfinite = 0;
  auto finish_cell = [&](int i, LP x, double uk) {
    double un;
    if constexpr (sizeof(LP) == 8)
      un = uk + (double)x;
    else
      un = f64_add_f32(uk, (float)x);
    const size_t idx = (size_t)i * nx + col;
    unew[idx] = un;
    if (vout) vout[idx] = to_f64(x);
    LP ru = rel_update(x, uk);
    if (!(ru <= err)) err = ru;
    if (!positive_finite_bits(un)) nonfinite = 1;
    const unsigned long long ub = (unsigned long long)__double_as_longlong(un);
    if (!(ub >> 63) && ub < hmin_bits) hmin_bits = ub;
    mass += fixed36_of_f64(un);
  };
  if (work && nch > 0) {
    issue_bw(nch - 1, 0);
    int it = 0;
    for (int q = nch - 1; q >= 0; --q, ++it) {
      const int buf = it & 1;
      if (q - 1 >= 0) {
        issue_bw(q - 1, buf ^ 1);
        __pipeline_wait_prior(1);
      } else {
        __pipeline_wait_prior(0);
      }
      __syncwarp();
      const int r0 = chunk_r0(q), r1 = chunk_r1(q);
      if (active) {
        if (half == 0) {
          for (int i = r1 - 1; i >= r0; --i) {
            const int k = i - r0;
            LP x = (twisted && i >= m - 2)
                       ? S.xs[lane][i - (m - 2)]
                       : W.st.bw.f[buf][2][k][lane] - W.st.bw.f[buf][0][k][lane] * x1 -
                             W.st.bw.f[buf][1][k][lane] * x2;
            x2 = x1;
            x1 = x;
            finish_cell(i, x, W.st.bw.u[buf][k][lane]);
          }
        } else {
          for (int i = r0; i < r1; ++i) {
            const int k = i - r0;
            LP x = (i <= m + 1) ? S.xs[lane][i - (m - 2)]
                                : W.st.bw.f[buf][2][k][lane] - W.st.bw.f[buf][0][k][lane] * x1 -
                                      W.st.bw.f[buf][1][k][lane] * x2;
            x2 = x1;
            x1 = x;
            finish_cell(i, x, W.st.bw.u[buf][k][lane]);
          }
        }
      }
      __syncwarp();
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    LP e2 = __shfl_xor_sync(0xffffffffu, err, o);
    if (!(e2 <= err)) err = e2;
    unsigned long long h2 = __shfl_xor_sync(0xffffffffu, hmin_bits, o);
    if (h2 < hmin_bits) hmin_bits = h2;
    mass += __shfl_xor_sync(0xffffffffu, mass, o);
    nonfinite |= __shfl_xor_sync(0xffffffffu, nonfinite, o);
    pivot_bad |= __shfl_xor_sync(0xffffffffu, pivot_bad, o);
  }
  if (lane == 0) {
    PartY p;
    p.err = (double)err;
    p.hmin = __longlong_as_double((long long)hmin_bits);
    p.mass = mass;
    p.nonfinite = nonfinite;
    p.pivot = pivot_bad;
    S.part[half] = p;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    PartY a = S.part[0], b = S.part[1];
    if (!(b.err <= a.err)) a.err = b.err;
    a.hmin = fmin(a.hmin, b.hmin);
    a.mass += b.mass;
    a.nonfinite |= b.nonfinite;
    a.pivot |= b.pivot;
    part[blockIdx.x] = a;
  }
}

}  // namespace tf
