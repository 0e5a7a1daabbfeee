// tf_line_sweeps.cuh -- warp-specialised line sweeps.
//
// The exact twisted LU solve of every line (see tf_sweeps.cuh) has a short
// sequential recurrence per cell; everything else per cell (the film values,
// the face derivatives of the fluxes, the band of the row, the right side,
// the Newton update and the reductions) has no loop-carried dependence.
// These kernels split the two: per block, SOLVER warps (one per half-line
// group) run only the recurrences, while PRODUCER warps compute the band rows
// of the next chunk into shared memory, stage tiles with cp.async, and, on
// the way back, apply the update and the reductions to the chunk the solvers
// just finished.  All warps advance in lockstep ticks separated by block
// barriers, so a chunk's band is produced one tick before it is solved.
#pragma once

#include "tf_sweeps.cuh"

namespace tf {

constexpr int kRY = 12;      // rows per chunk of the y sweep (4 groups of 3)
constexpr int kCX = 12;      // columns per chunk of the x sweep
constexpr int kProd = 8;     // producer warps per block
constexpr int kSweepThreads = 32 * (2 + kProd);

// Band of line cell j from its two faces (natural orientation):
// a..e multiply x_{j-2}..x_{j+2}.

constexpr int kNP = 32 * kProd;  // producer threads

// Film value of a tile in LP (the FP32 Jacobian needs the truncated height).
template <class LP> __device__ __forceinline__ LP tile_lp(double u);
template <> __device__ __forceinline__ double tile_lp<double>(double u) { return u; }
template <> __device__ __forceinline__ float tile_lp<float>(double u) { return f32_of_pos_f64_fast(u); }

// Copy an R x C tile of u with top-left corner (row0, col0) into shared
// memory (row pitch DP), reflecting indices at the walls; tiles that touch
// no wall take the plain path.  Executed by the producer threads.
template <int R, int C, int DP>
__device__ __forceinline__ void copy_tile_f64(double* dst, const double* __restrict__ u, int row0,
                                              int col0, int ny, int nx, int p) {
  const bool inner = row0 >= 0 && row0 + R <= ny && col0 >= 0 && col0 + C <= nx;
  if (inner) {
    const double* base = u + (size_t)row0 * nx + col0;
    for (int k = p; k < R * C; k += kNP) {
      const int r = k / C, c = k - r * C;
      cp8(dst + r * DP + c, base + (size_t)r * nx + c);
    }
  } else {
    for (int k = p; k < R * C; k += kNP) {
      const int r = k / C, c = k - r * C;
      const int gj = reflect_index(row0 + r, ny), gi = reflect_index(col0 + c, nx);
      cp8(dst + r * DP + c, u + (size_t)gj * nx + gi);
    }
  }
}

// Per-cell film values, pre-scaled for the band: with k3 = theta dt/(2 ds^4)
// and k1 = theta dt/(2 ds^2),
//   F0 = k3 f0, F1 = k1 f1, D0 = k1 f0', D1 = k1 f1',
// so that for the face between line cells p and q (the scaled dF of
// face_dF): c3 = F0_p + F0_q, Bd = F1_p + F1_q,
//   t_p = D0_p (lap_q - lap_p) + D1_p (u_q - u_p), t_q likewise, and
//   dF = (-w_p c3, (2 + w_p) c3 + t_p - Bd, -(2 + w_q) c3 + t_q + Bd, w_q c3).
template <class LP> struct CellS {
  LP u, lap, F0, F1, D0, D1;
};

template <class LP, class Acc>
__device__ __forceinline__ CellS<LP> cell_scaled(const MobC<LP>& ml, LP inv_ds2, LP k3, LP k1, Acc U) {
  CellS<LP> X;
  const LP uc = U(0, 0);
  X.u = uc;
  X.lap = (((U(0, 1) - uc) + (U(0, -1) - uc)) + ((U(1, 0) - uc) + (U(-1, 0) - uc))) * inv_ds2;
  const LP s = rcp(uc);
  LP f0, f1, d0, d1;
  mobility(ml, uc, s, f0, f1);
  mobility_d(ml, uc, s, d0, d1);
  X.F0 = k3 * f0;
  X.F1 = k1 * f1;
  X.D0 = k1 * d0;
  X.D1 = k1 * d1;
  return X;
}

template <class LP>
__device__ __forceinline__ void face_scaled(const CellS<LP>& P, const CellS<LP>& Q, bool pl, bool qr,
                                            LP dF[4]) {
  const LP dl = Q.lap - P.lap, du = Q.u - P.u;
  const LP c3 = P.F0 + Q.F0, Bd = P.F1 + Q.F1;
  const LP tp = P.D0 * dl + P.D1 * du, tq = Q.D0 * dl + Q.D1 * du;
  if (pl && qr) {
    dF[0] = -c3;
    dF[1] = LP(3) * c3 + (tp - Bd);
    dF[2] = LP(-3) * c3 + (tq + Bd);
    dF[3] = c3;
  } else {
    const LP wp = pl ? LP(1) : LP(0), wq = qr ? LP(1) : LP(0);
    dF[0] = -wp * c3;
    dF[1] = (LP(2) + wp) * c3 + (tp - Bd);
    dF[2] = -(LP(2) + wq) * c3 + (tq + Bd);
    dF[3] = wq * c3;
  }
}

// Struct-of-arrays cell buffer: scaled film values of the cells of one chunk
// plus one halo cell at each end, for 32 lines: [field][cell][line].
template <class LP, int L> struct CellBuf {
  LP v[6][L + 2][32];
  __device__ __forceinline__ void put(int cell, int line, const CellS<LP>& X) {
    v[0][cell][line] = X.u;
    v[1][cell][line] = X.lap;
    v[2][cell][line] = X.F0;
    v[3][cell][line] = X.F1;
    v[4][cell][line] = X.D0;
    v[5][cell][line] = X.D1;
  }
  __device__ __forceinline__ CellS<LP> get(int cell, int line) const {
    CellS<LP> X;
    X.u = v[0][cell][line];
    X.lap = v[1][cell][line];
    X.F0 = v[2][cell][line];
    X.F1 = v[3][cell][line];
    X.D0 = v[4][cell][line];
    X.D1 = v[5][cell][line];
    return X;
  }
};

// Band rows of cells [ia, ib) of one line (chunk origin c0, line length n)
// from the cell buffer (cell i at index i - c0 + 1), written to B[f][i-c0][line]
// with the right side r taken from R(i).
template <class LP, int L, class RhsF>
__device__ __forceinline__ void band_group(const CellBuf<LP, L>& cb, int line, int c0, int ia, int ib,
                                           int n, LP* B, RhsF R) {
  CellS<LP> P = cb.get(ia - c0 + 1, line);
  LP Lf[4] = {LP(0), LP(0), LP(0), LP(0)};
  if (ia > 0) face_scaled(cb.get(ia - c0, line), P, ia - 1 > 0, ia + 1 < n, Lf);
  for (int i = ia; i < ib; ++i) {
    LP Rf[4] = {LP(0), LP(0), LP(0), LP(0)};
    if (i + 1 < n) {
      CellS<LP> Q = cb.get(i - c0 + 2, line);
      face_scaled(P, Q, i > 0, i + 2 < n, Rf);
      P = Q;
    }
    const int k = (i - c0) * 32 + line;
    B[0 * L * 32 + k] = -Lf[0];
    B[1 * L * 32 + k] = Rf[0] - Lf[1];
    B[2 * L * 32 + k] = LP(1) + (Rf[1] - Lf[2]);
    B[3 * L * 32 + k] = Rf[2] - Lf[3];
    B[4 * L * 32 + k] = Rf[3];
    B[5 * L * 32 + k] = R(i);
    for (int q = 0; q < 4; ++q) Lf[q] = Rf[q];
  }
}

// ---------------------------------------------------------------------------
// y sweep.  Block: 32 columns i0..i0+31.  Warp 0 / 1 solve the top / bottom
// halves; warps 2..5 produce.  Producer thread p: half = p >> 6,
// col = p & 31, row group = (p >> 5) & 1 (8 rows of a 16-row chunk).

template <class LP> struct YFwd {
  double ut[2][2][kRY + 4][34];  // raw film tiles (rows r0-2.., cols i0-1..)
  LP wt[2][2][kRY][32];          // right sides w
  LP lt[2][kRY + 4][35];         // film tile in LP (current producer chunk)
  LP band[2][2][6][kRY][32];     // [stage][half][a..e, r][row][col]
  CellBuf<LP, kRY> cb[2];        // film values of the chunk's cells
};
template <class LP> struct YBwd {
  LP ft[3][2][3][kRY][32];       // factor tiles
  double ukt[3][2][kRY][32];     // u_k tiles for the update
  LP xb[2][2][kRY][32];          // solved corrections
};
template <class LP> struct YSmem {
  union {
    YFwd<LP> f;
    YBwd<LP> b;
  } s;
  LUState<LP> seamS[32], seamR[32];
  LP xs[32][4];
  PartY part[kSweepThreads / 32];
};

template <class Mode>
__global__ void __launch_bounds__(kSweepThreads)
    k_ysweep(ModelK M, StepK K, const double* __restrict__ u, const typename Mode::LP* __restrict__ w,
              typename Mode::LP* __restrict__ fac, double* __restrict__ unew,
              double* __restrict__ vout, PartY* __restrict__ part) {
  typedef typename Mode::LP LP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  YSmem<LP>& S = *reinterpret_cast<YSmem<LP>*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool solver = warp < 2;
  const int p = threadIdx.x - 64;  // producer index (valid when !solver)
  const int nx = M.nx, ny = M.ny;
  const size_t N = (size_t)nx * ny;
  const int i0 = blockIdx.x * 32;
  const int m = split_point(ny);
  const bool twisted = m < ny;
  const int nchh[2] = {(m + kRY - 1) / kRY, twisted ? (ny - m + kRY - 1) / kRY : 0};
  const int nch = max(nchh[0], nchh[1]);
  auto r0_of = [&](int h, int q) { return h == 0 ? q * kRY : max(m, ny - (q + 1) * kRY); };
  auto r1_of = [&](int h, int q) { return h == 0 ? min(m, (q + 1) * kRY) : ny - q * kRY; };
  const MobC<LP> ml = mob_consts<LP>(M);
  const LP inv_ds2 = (LP)M.inv_ds2;
  const LP k3 = (LP)(0.5 * K.theta_dt * M.inv_ds3 * M.inv_ds);
  const LP k1 = (LP)(0.5 * K.theta_dt * M.inv_ds2);
  LP* fg = fac;
  LP* fd = fac + N;
  LP* fz = fac + 2 * N;
  int pivot_bad = 0;

  // ---------------- producer helpers ----------------
  // issue the film and w tiles of chunk q of both halves into ring slot q & 1
  auto issue_fwd = [&](int q) {
    const int slot = q & 1;
    for (int h = 0; h < 2; ++h) {
      if (q >= nchh[h]) continue;
      const int r0 = r0_of(h, q), r1 = r1_of(h, q);
      copy_tile_f64<kRY + 4, 34, 34>(&S.s.f.ut[slot][h][0][0], u, r0 - 2, i0 - 1, ny, nx, p);
      for (int k = p; k < kRY * 32; k += kNP) {
        int r = k >> 5, c = k & 31;
        if (r0 + r < r1 && i0 + c < nx) cpT(&S.s.f.wt[slot][h][r][c], w + (size_t)(r0 + r) * nx + i0 + c);
      }
    }
    __pipeline_commit();
  };
  auto pbar = [&]() { asm volatile("bar.sync 1, %0;" ::"n"(kNP)); };

  LUState<LP> lu;
  lu.reset();

  // ---------------- forward ticks ----------------
  if (!solver) issue_fwd(0);
  for (int t = 0; t <= nch; ++t) {
    if (!solver) {
      if (t < nch) {
        __pipeline_wait_prior(0);  // chunk t landed (issued one tick ago)
        pbar();
        if (t + 1 < nch) issue_fwd(t + 1);  // slot (t+1)&1 was consumed last tick
        const int slot = t & 1;
        for (int h = 0; h < 2; ++h) {
          if (t >= nchh[h]) continue;
          for (int k = p; k < (kRY + 4) * 34; k += kNP) {
            int r = k / 34, c = k - r * 34;
            S.s.f.lt[h][r][c] = tile_lp<LP>(S.s.f.ut[slot][h][r][c]);
          }
        }
        pbar();
        // phase A: film values of rows r0-1..r1 of each half's 32 columns
        for (int h = 0; h < 2; ++h) {
          if (t >= nchh[h]) continue;
          const int r0 = r0_of(h, t), r1 = r1_of(h, t);
          for (int k = p; k < (kRY + 2) * 32; k += kNP) {
            const int cr = k >> 5, c = k & 31;  // cell row index: global row r0 - 1 + cr
            if (r0 - 1 + cr > r1 || i0 + c >= nx) continue;
            const int rr = cr + 1, cc = c + 1;  // tile position of the cell
            S.s.f.cb[h].put(cr, c, cell_scaled<LP>(ml, inv_ds2, k3, k1, [&](int dr, int dc) {
                              return S.s.f.lt[h][rr + dr][cc + dc];
                            }));
          }
        }
        pbar();
        // phase B: band rows; thread p covers (half, column, 3 rows)
        {
          const int h = p >> 7, g = (p >> 5) & 3, c = p & 31;
          if (t < nchh[h] && i0 + c < nx) {
            const int r0 = r0_of(h, t), r1 = r1_of(h, t);
            const int ja = r0 + 3 * g, jb = min(r1, ja + 3);
            if (ja < jb)
              band_group<LP, kRY>(S.s.f.cb[h], c, r0, ja, jb, ny, &S.s.f.band[t & 1][h][0][0][0],
                                  [&](int j) { return S.s.f.wt[slot][h][j - r0][c]; });
          }
        }
      }
    } else if (t >= 1) {
      const int q = t - 1, h = warp;
      if (q < nchh[h] && i0 + lane < nx) {
        const int r0 = r0_of(h, q), r1 = r1_of(h, q);
        const LP* B = &S.s.f.band[q & 1][h][0][0][0];
        const int col = i0 + lane;
        if (h == 0) {
          for (int j = r0; j < r1; ++j) {
            const int k = (j - r0) * 32 + lane;
            LP g, dl, z;
            if (!lu.step(B[k], B[kRY * 32 + k], B[2 * kRY * 32 + k], B[3 * kRY * 32 + k],
                         B[4 * kRY * 32 + k], B[5 * kRY * 32 + k], g, dl, z))
              pivot_bad = 1;
            const size_t idx = (size_t)j * nx + col;
            fg[idx] = g;
            fd[idx] = dl;
            fz[idx] = z;
          }
        } else {
          for (int j = r1 - 1; j >= r0; --j) {
            const int k = (j - r0) * 32 + lane;
            LP g, dl, z;
            if (!lu.step(B[4 * kRY * 32 + k], B[3 * kRY * 32 + k], B[2 * kRY * 32 + k],
                         B[kRY * 32 + k], B[k], B[5 * kRY * 32 + k], g, dl, z))
              pivot_bad = 1;
            const size_t idx = (size_t)j * nx + col;
            fg[idx] = g;
            fd[idx] = dl;
            fz[idx] = z;
          }
        }
      }
    }
    __syncthreads();
  }
  // ---------------- seam ----------------
  if (warp == 0) S.seamS[lane] = lu;
  if (warp == 1) S.seamR[lane] = lu;
  __syncthreads();
  if (warp == 0 && twisted) {
    LP x[4] = {LP(0), LP(0), LP(0), LP(0)};
    if (!seam(S.seamS[lane], S.seamR[lane], x) && i0 + lane < nx) pivot_bad = 1;
    for (int q = 0; q < 4; ++q) S.xs[lane][q] = x[q];
  }
  __syncthreads();

  // ---------------- backward ticks ----------------
  // chunk order: b-th backward chunk of half h is chunk nchh[h]-1-b.
  auto issue_bwd_f = [&](int bq) {  // factor tiles of backward chunk bq
    const int slot = bq % 3;
    for (int h = 0; h < 2; ++h) {
      const int q = nchh[h] - 1 - bq;
      if (q < 0) continue;
      const int r0 = r0_of(h, q), r1 = r1_of(h, q);
      for (int k = p; k < 3 * kRY * 32; k += kNP) {
        int f = k / (kRY * 32), rem = k - f * kRY * 32, r = rem >> 5, c = rem & 31;
        if (r0 + r < r1 && i0 + c < nx)
          cpT(&S.s.b.ft[slot][h][f][r][c], fac + (size_t)f * N + (size_t)(r0 + r) * nx + i0 + c);
      }
    }
  };
  auto issue_bwd_u = [&](int bq) {  // u_k tiles of backward chunk bq
    const int slot = bq % 3;
    for (int h = 0; h < 2; ++h) {
      const int q = nchh[h] - 1 - bq;
      if (q < 0) continue;
      const int r0 = r0_of(h, q), r1 = r1_of(h, q);
      for (int k = p; k < kRY * 32; k += kNP) {
        int r = k >> 5, c = k & 31;
        if (r0 + r < r1 && i0 + c < nx)
          cp8(&S.s.b.ukt[slot][h][r][c], u + (size_t)(r0 + r) * nx + i0 + c);
      }
    }
  };
  LP x1 = LP(0), x2 = LP(0);
  if (solver && twisted) {
    if (warp == 0) {
      x1 = S.xs[lane][2];
      x2 = S.xs[lane][3];
    } else {
      x1 = S.xs[lane][1];
      x2 = S.xs[lane][0];
    }
  }
  // per-iteration reductions: the Newton test and positivity (mass and min h
  // of the accepted film are reduced once per step by k_grid_stats)
  LP err = LP(0);
  int nonfinite = 0;
  // cp.async groups: before the ticks {f0, u0} and {f1}; tick t issues
  // {f(t+2), u(t+1)} and then waits for everything older, so the solvers
  // find f(t+1) and the producers find u(t) at tick t+1.
  if (!solver) {
    issue_bwd_f(0);
    issue_bwd_u(0);
    __pipeline_commit();
    if (nch > 1) issue_bwd_f(1);
    __pipeline_commit();
    __pipeline_wait_prior(1);  // backward chunk 0 ready for the solvers
  }
  __syncthreads();
  for (int t = 0; t <= nch; ++t) {
    if (solver) {
      if (t < nch) {
        const int h = warp, q = nchh[h] - 1 - t;
        if (q >= 0 && i0 + lane < nx) {
          const int r0 = r0_of(h, q), r1 = r1_of(h, q);
          const int slot = t % 3;
          LP* X = &S.s.b.xb[t & 1][h][0][0];
          if (h == 0) {
            for (int j = r1 - 1; j >= r0; --j) {
              const int k = j - r0;
              LP x = (twisted && j >= m - 2)
                         ? S.xs[lane][j - (m - 2)]
                         : S.s.b.ft[slot][h][2][k][lane] - S.s.b.ft[slot][h][0][k][lane] * x1 -
                               S.s.b.ft[slot][h][1][k][lane] * x2;
              x2 = x1;
              x1 = x;
              X[k * 32 + lane] = x;
            }
          } else {
            for (int j = r0; j < r1; ++j) {
              const int k = j - r0;
              LP x = (j <= m + 1) ? S.xs[lane][j - (m - 2)]
                                  : S.s.b.ft[slot][h][2][k][lane] - S.s.b.ft[slot][h][0][k][lane] * x1 -
                                        S.s.b.ft[slot][h][1][k][lane] * x2;
              x2 = x1;
              x1 = x;
              X[k * 32 + lane] = x;
            }
          }
        }
      }
    } else {
      // finish backward chunk t-1: update, store, reduce
      if (t >= 1) {
        const int bq = t - 1, slot = bq % 3;
        for (int h = 0; h < 2; ++h) {
          const int q = nchh[h] - 1 - bq;
          if (q < 0) continue;
          const int r0 = r0_of(h, q), r1 = r1_of(h, q);
          const LP* X = &S.s.b.xb[bq & 1][h][0][0];
          for (int k = p; k < kRY * 32; k += kNP) {
            int r = k >> 5, c = k & 31;
            const int j = r0 + r, col = i0 + c;
            if (j >= r1 || col >= nx) continue;
            const LP x = X[k];
            const double uk = S.s.b.ukt[slot][h][r][c];
            double un;
            if constexpr (sizeof(LP) == 8)
              un = uk + (double)x;
            else
              un = f64_add_f32(uk, (float)x);
            const size_t idx = (size_t)j * nx + col;
            unew[idx] = un;
            if (vout) vout[idx] = to_f64(x);
            LP ru = rel_update(x, uk);
            if (!(ru <= err)) err = ru;
            if (!positive_finite_bits(un)) nonfinite = 1;
          }
        }
      }
      // prefetch: factors two chunks ahead, u_k one chunk ahead of the solvers
      if (t + 2 < nch) issue_bwd_f(t + 2);
      if (t + 1 < nch) issue_bwd_u(t + 1);
      __pipeline_commit();
      __pipeline_wait_prior(1);
    }
    __syncthreads();
  }
  // ---------------- block reduction ----------------
  for (int o = 16; o > 0; o >>= 1) {
    LP e2 = __shfl_xor_sync(0xffffffffu, err, o);
    if (!(e2 <= err)) err = e2;
    nonfinite |= __shfl_xor_sync(0xffffffffu, nonfinite, o);
    pivot_bad |= __shfl_xor_sync(0xffffffffu, pivot_bad, o);
  }
  if (lane == 0) {
    PartY pp;
    pp.err = (double)err;
    pp.hmin = INFINITY;
    pp.mass = 0;
    pp.nonfinite = nonfinite;
    pp.pivot = pivot_bad;
    S.part[warp] = pp;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    PartY a = S.part[0];
    for (int k = 1; k < kSweepThreads / 32; ++k) {
      const PartY& b = S.part[k];
      if (!(b.err <= a.err)) a.err = b.err;
      if (b.hmin < a.hmin) a.hmin = b.hmin;
      a.mass += b.mass;
      a.nonfinite |= b.nonfinite;
      a.pivot |= b.pivot;
    }
    part[blockIdx.x] = a;
  }
}

// ---------------------------------------------------------------------------
// x sweep.  Block: 32 rows j0..j0+31.  Warp 0 / 1 solve the left / right
// halves of the rows (lane = row); warps 2..5 produce.  Producer thread p:
// half = p >> 6, row = p & 31, column group = (p >> 5) & 1 (8 columns of a
// 16-column chunk).  Factor scratch per block: fac[((blk*3 + f)*nx + col)*32 + row].

template <class LP> struct XFwd {
  double ut[2][2][34][kCX + 4];  // raw film tiles (rows j0-1.., cols c0-2..)
  LP rt[2][2][32][kCX + 1];      // right sides
  LP lt[2][34][kCX + 5];         // film tile in LP
  LP band[2][2][6][kCX][32];     // [stage][half][a..e, r][col][row]
  CellBuf<LP, kCX> cb[2];        // film values of the chunk's cells
};
template <class LP> struct XBwd {
  LP ft[3][2][3][kCX][32];       // factor tiles [f][col][row]
  LP xb[2][2][kCX][33];          // solved w [col][row]
};
template <class LP> struct XSmem {
  union {
    XFwd<LP> f;
    XBwd<LP> b;
  } s;
  LUState<LP> seamS[32], seamR[32];
  LP xs[32][4];
  int piv[kSweepThreads / 32];
};

template <class Mode>
__global__ void __launch_bounds__(kSweepThreads)
    k_xsweep(ModelK M, StepK K, const double* __restrict__ u, typename Mode::LP* __restrict__ rw,
              typename Mode::LP* __restrict__ fac, PartX* __restrict__ part) {
  typedef typename Mode::LP LP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  XSmem<LP>& S = *reinterpret_cast<XSmem<LP>*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool solver = warp < 2;
  const int p = threadIdx.x - 64;
  const int nx = M.nx, ny = M.ny;
  const int j0 = blockIdx.x * 32;
  const int m = split_point(nx);
  const bool twisted = m < nx;
  const int nchh[2] = {(m + kCX - 1) / kCX, twisted ? (nx - m + kCX - 1) / kCX : 0};
  const int nch = max(nchh[0], nchh[1]);
  auto c0_of = [&](int h, int q) { return h == 0 ? q * kCX : max(m, nx - (q + 1) * kCX); };
  auto c1_of = [&](int h, int q) { return h == 0 ? min(m, (q + 1) * kCX) : nx - q * kCX; };
  const MobC<LP> ml = mob_consts<LP>(M);
  const LP inv_ds2 = (LP)M.inv_ds2;
  const LP k3 = (LP)(0.5 * K.theta_dt * M.inv_ds3 * M.inv_ds);
  const LP k1 = (LP)(0.5 * K.theta_dt * M.inv_ds2);
  LP* facb = fac + (size_t)blockIdx.x * 3 * nx * 32;
  int pivot_bad = 0;

  auto issue_fwd = [&](int q) {
    const int slot = q & 1;
    for (int h = 0; h < 2; ++h) {
      if (q >= nchh[h]) continue;
      const int c0 = c0_of(h, q), c1 = c1_of(h, q);
      copy_tile_f64<34, kCX + 4, kCX + 4>(&S.s.f.ut[slot][h][0][0], u, j0 - 1, c0 - 2, ny, nx, p);
      for (int k = p; k < 32 * kCX; k += kNP) {
        int r = k / kCX, c = k - r * kCX;
        if (j0 + r < ny && c0 + c < c1) cpT(&S.s.f.rt[slot][h][r][c], rw + (size_t)(j0 + r) * nx + c0 + c);
      }
    }
    __pipeline_commit();
  };
  auto pbar = [&]() { asm volatile("bar.sync 1, %0;" ::"n"(kNP)); };

  LUState<LP> lu;
  lu.reset();
  if (!solver) issue_fwd(0);
  for (int t = 0; t <= nch; ++t) {
    if (!solver) {
      if (t < nch) {
        __pipeline_wait_prior(0);  // chunk t landed (issued one tick ago)
        pbar();
        if (t + 1 < nch) issue_fwd(t + 1);  // slot (t+1)&1 was consumed last tick
        const int slot = t & 1;
        for (int h = 0; h < 2; ++h) {
          if (t >= nchh[h]) continue;
          for (int k = p; k < 34 * (kCX + 4); k += kNP) {
            int r = k / (kCX + 4), c = k - r * (kCX + 4);
            S.s.f.lt[h][r][c] = tile_lp<LP>(S.s.f.ut[slot][h][r][c]);
          }
        }
        pbar();
        // phase A: film values of cols c0-1..c1 of each half's 32 rows
        for (int h = 0; h < 2; ++h) {
          if (t >= nchh[h]) continue;
          const int c0 = c0_of(h, t), c1 = c1_of(h, t);
          for (int k = p; k < (kCX + 2) * 32; k += kNP) {
            const int ci = k >> 5, r = k & 31;  // cell col index: global col c0 - 1 + ci
            if (c0 - 1 + ci > c1 || j0 + r >= ny) continue;
            const int rr = r + 1, cc = ci + 1;
            S.s.f.cb[h].put(ci, r, cell_scaled<LP>(ml, inv_ds2, k3, k1, [&](int dr, int dc) {
                              return S.s.f.lt[h][rr + dr][cc + dc];
                            }));
          }
        }
        pbar();
        // phase B: band rows; thread p covers (half, row, 3 columns)
        {
          const int h = p >> 7, g = (p >> 5) & 3, r = p & 31;
          if (t < nchh[h] && j0 + r < ny) {
            const int c0 = c0_of(h, t), c1 = c1_of(h, t);
            const int ia = c0 + 3 * g, ib = min(c1, ia + 3);
            if (ia < ib)
              band_group<LP, kCX>(S.s.f.cb[h], r, c0, ia, ib, nx, &S.s.f.band[t & 1][h][0][0][0],
                                  [&](int i) { return S.s.f.rt[slot][h][r][i - c0]; });
          }
        }
      }
    } else if (t >= 1) {
      const int q = t - 1, h = warp;
      if (q < nchh[h] && j0 + lane < ny) {
        const int c0 = c0_of(h, q), c1 = c1_of(h, q);
        const LP* B = &S.s.f.band[q & 1][h][0][0][0];
        LP* fg = facb;
        LP* fd = facb + (size_t)nx * 32;
        LP* fz = facb + (size_t)2 * nx * 32;
        if (h == 0) {
          for (int i = c0; i < c1; ++i) {
            const int k = (i - c0) * 32 + lane;
            LP g, dl, z;
            if (!lu.step(B[k], B[kCX * 32 + k], B[2 * kCX * 32 + k], B[3 * kCX * 32 + k],
                         B[4 * kCX * 32 + k], B[5 * kCX * 32 + k], g, dl, z))
              pivot_bad = 1;
            fg[(size_t)i * 32 + lane] = g;
            fd[(size_t)i * 32 + lane] = dl;
            fz[(size_t)i * 32 + lane] = z;
          }
        } else {
          for (int i = c1 - 1; i >= c0; --i) {
            const int k = (i - c0) * 32 + lane;
            LP g, dl, z;
            if (!lu.step(B[4 * kCX * 32 + k], B[3 * kCX * 32 + k], B[2 * kCX * 32 + k],
                         B[kCX * 32 + k], B[k], B[5 * kCX * 32 + k], g, dl, z))
              pivot_bad = 1;
            fg[(size_t)i * 32 + lane] = g;
            fd[(size_t)i * 32 + lane] = dl;
            fz[(size_t)i * 32 + lane] = z;
          }
        }
      }
    }
    __syncthreads();
  }
  if (warp == 0) S.seamS[lane] = lu;
  if (warp == 1) S.seamR[lane] = lu;
  __syncthreads();
  if (warp == 0 && twisted) {
    LP x[4] = {LP(0), LP(0), LP(0), LP(0)};
    if (!seam(S.seamS[lane], S.seamR[lane], x) && j0 + lane < ny) pivot_bad = 1;
    for (int q = 0; q < 4; ++q) S.xs[lane][q] = x[q];
  }
  __syncthreads();
  auto issue_bwd = [&](int bq) {
    const int slot = bq % 3;
    for (int h = 0; h < 2; ++h) {
      const int q = nchh[h] - 1 - bq;
      if (q < 0) continue;
      const int c0 = c0_of(h, q), c1 = c1_of(h, q);
      for (int f = 0; f < 3; ++f) {
        const LP* src = facb + ((size_t)f * nx + c0) * 32;
        for (int k = p; k < (c1 - c0) * 32; k += kNP)
          cpT(&S.s.b.ft[slot][h][f][k >> 5][k & 31], src + k);
      }
    }
    __pipeline_commit();
  };
  LP x1 = LP(0), x2 = LP(0);
  if (solver && twisted) {
    if (warp == 0) {
      x1 = S.xs[lane][2];
      x2 = S.xs[lane][3];
    } else {
      x1 = S.xs[lane][1];
      x2 = S.xs[lane][0];
    }
  }
  if (!solver) {
    issue_bwd(0);
    if (nch > 1) issue_bwd(1);
    else __pipeline_commit();
    __pipeline_wait_prior(1);
  }
  __syncthreads();
  for (int t = 0; t <= nch; ++t) {
    if (solver) {
      if (t < nch) {
        const int h = warp, q = nchh[h] - 1 - t;
        if (q >= 0 && j0 + lane < ny) {
          const int c0 = c0_of(h, q), c1 = c1_of(h, q);
          const int slot = t % 3;
          if (h == 0) {
            for (int i = c1 - 1; i >= c0; --i) {
              const int k = i - c0;
              LP x = (twisted && i >= m - 2)
                         ? S.xs[lane][i - (m - 2)]
                         : S.s.b.ft[slot][h][2][k][lane] - S.s.b.ft[slot][h][0][k][lane] * x1 -
                               S.s.b.ft[slot][h][1][k][lane] * x2;
              x2 = x1;
              x1 = x;
              S.s.b.xb[t & 1][h][k][lane] = x;
            }
          } else {
            for (int i = c0; i < c1; ++i) {
              const int k = i - c0;
              LP x = (i <= m + 1) ? S.xs[lane][i - (m - 2)]
                                  : S.s.b.ft[slot][h][2][k][lane] - S.s.b.ft[slot][h][0][k][lane] * x1 -
                                        S.s.b.ft[slot][h][1][k][lane] * x2;
              x2 = x1;
              x1 = x;
              S.s.b.xb[t & 1][h][k][lane] = x;
            }
          }
        }
      }
    } else {
      if (t >= 1) {  // store w of backward chunk t-1, coalesced along rows
        const int bq = t - 1;
        for (int h = 0; h < 2; ++h) {
          const int q = nchh[h] - 1 - bq;
          if (q < 0) continue;
          const int c0 = c0_of(h, q), c1 = c1_of(h, q);
          for (int k = p; k < 32 * kCX; k += kNP) {
            int r = k / kCX, c = k - r * kCX;
            if (j0 + r < ny && c0 + c < c1) rw[(size_t)(j0 + r) * nx + c0 + c] = S.s.b.xb[bq & 1][h][c][r];
          }
        }
      }
      if (t + 2 < nch) issue_bwd(t + 2);
      else __pipeline_commit();
      __pipeline_wait_prior(1);
    }
    __syncthreads();
  }
  const int pv = __any_sync(0xffffffffu, pivot_bad);
  if (lane == 0) S.piv[warp] = pv;
  __syncthreads();
  if (threadIdx.x == 0) {
    int a = 0;
    for (int k = 0; k < kSweepThreads / 32; ++k) a |= S.piv[k];
    PartX pp;
    pp.gnorm = 0.0;
    pp.pivot = a;
    pp.pad = 0;
    part[blockIdx.x] = pp;
  }
}

}  // namespace tf
