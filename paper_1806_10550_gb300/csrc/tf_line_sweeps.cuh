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

constexpr int kRY = 24;      // rows per chunk of the y sweep
constexpr int kCX = 24;      // columns per chunk of the x sweep
constexpr int kG = 6;        // cells of a chunk whose band rows one producer thread builds
constexpr int kProd = 8;     // producer warps per block
constexpr int kSweepThreads = 32 * (2 + kProd);

// Band of line cell j from its two faces (natural orientation):
// a..e multiply x_{j-2}..x_{j+2}.

constexpr int kNP = 32 * kProd;  // producer threads
static_assert(2 * 4 * 32 == kNP && 4 * kG == kRY && 4 * kG == kCX,
              "each producer thread owns one group of kG cells of one line half");

// Tile copies into shared memory, executed by the kNP producer threads.  The
// fast paths give every thread a fixed, compile-time set of elements (no
// loop bookkeeping per element); the rare paths (wall reflection, unaligned
// rows) stay rolled to keep the kernels' code small.

// Interior rows [0, nr) x C columns starting at base (row pitch `pitch`
// elements) in 16-byte vectors: base and pitch 16-byte aligned, C and DP
// multiples of a vector.
template <class T, int R, int C, int DP>
__device__ __forceinline__ void copy_rows_vec(T* dst, const T* __restrict__ base, size_t pitch, int nr,
                                              int p) {
  constexpr int V = 16 / sizeof(T), CV = C / V, NI = (R * CV + kNP - 1) / kNP;
  static_assert(C % V == 0 && DP % V == 0, "vector copies need whole vectors");
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    const int k = p + i * kNP;
    const int r = k / CV, c = (k - r * CV) * V;
    if (k < R * CV && r < nr) __pipeline_memcpy_async(dst + r * DP + c, base + r * pitch + c, 16);
  }
}

// Interior rows [0, nr) x columns [0, nc) (nc <= C <= 32) element by element,
// the 32 lanes of a warp along a row (coalesced), eight row groups.
template <class T, int R, int C, int DP>
__device__ __forceinline__ void copy_rows_elem(T* dst, const T* __restrict__ base, size_t pitch, int nr,
                                               int nc, int p) {
  static_assert(C <= 32 && kNP == 256, "one warp per row, eight row groups");
  const int c = p & 31, rg = p >> 5;
  if (c >= nc) return;
#pragma unroll
  for (int i = 0; i < (R + 7) / 8; ++i) {
    const int r = rg + 8 * i;
    if (r < nr) cpT(dst + r * DP + c, base + r * pitch + c);
  }
}

// An R x C tile of a row-major [ny][nx] array with top-left corner
// (row0, col0), indices reflected at the walls.
template <class T, int R, int C, int DP>
__device__ __forceinline__ void copy_tile(T* dst, const T* __restrict__ src, int row0, int col0, int ny,
                                          int nx, int p) {
  constexpr int V = 16 / sizeof(T);
  const bool inner = row0 >= 0 && row0 + R <= ny && col0 >= 0 && col0 + C <= nx;
  const T* base = src + (size_t)row0 * nx + col0;
  if constexpr ((C % V) == 0 && (DP % V) == 0) {
    if (inner && (nx % V) == 0 && (reinterpret_cast<uintptr_t>(base) & 15) == 0) {
      copy_rows_vec<T, R, C, DP>(dst, base, nx, R, p);
      return;
    }
  }
  if constexpr (C <= 32) {
    if (inner) {
      copy_rows_elem<T, R, C, DP>(dst, base, nx, R, C, p);
      return;
    }
  }
#pragma unroll 1
  for (int k = p; k < R * C; k += kNP) {
    const int r = k / C, c = k - r * C;
    const int gj = reflect_index(row0 + r, ny), gi = reflect_index(col0 + c, nx);
    cpT(dst + r * DP + c, src + (size_t)gj * nx + gi);
  }
}

// Rows [0, nr) x columns [0, C) of a row-major array (row stride nx) from
// (row0, col0), without reflection; columns at or beyond nx are skipped.
template <class T, int R, int C, int DP>
__device__ __forceinline__ void copy_rows(T* dst, const T* __restrict__ src, int row0, int col0, int nr,
                                          int nx, int p) {
  constexpr int V = 16 / sizeof(T);
  const T* base = src + (size_t)row0 * nx + col0;
  if constexpr ((C % V) == 0 && (DP % V) == 0) {
    if (col0 + C <= nx && (nx % V) == 0 && (reinterpret_cast<uintptr_t>(base) & 15) == 0) {
      copy_rows_vec<T, R, C, DP>(dst, base, nx, nr, p);
      return;
    }
  }
  if constexpr (C <= 32) {
    copy_rows_elem<T, R, C, DP>(dst, base, nx, nr, min(C, nx - col0), p);
  } else {
#pragma unroll 1
    for (int k = p; k < nr * C; k += kNP) {
      const int r = k / C, c = k - r * C;
      if (col0 + c < nx) cpT(dst + r * DP + c, base + (size_t)r * nx + c);
    }
  }
}

// n <= NMAX contiguous elements; 16-byte vectors when both ends are aligned.
template <class T, int NMAX>
__device__ __forceinline__ void copy_span(T* dst, const T* __restrict__ src, int n, int p) {
  constexpr int V = 16 / sizeof(T), NI = (NMAX / V + kNP - 1) / kNP;
  if ((n % V) == 0 && ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0) {
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      const int k = p + i * kNP;
      if (k < n / V) __pipeline_memcpy_async(dst + k * V, src + k * V, 16);
    }
  } else {
#pragma unroll 1
    for (int k = p; k < n; k += kNP) cpT(dst + k, src + k);
  }
}

// The Newton update's correction as a double, exactly: integer operations
// for an FP32 correction (f64_of_f32_exact), so that the update's one FP64
// add per cell is the backward ticks' only FP64-pipe work
__device__ __forceinline__ double widen_exact(float x) { return f64_of_f32_exact(x); }
__device__ __forceinline__ double widen_exact(double x) { return x; }

// a * b rounded on its own: never contracted with a following add
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

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
  mobility_all(ml, uc, s, f0, f1, d0, d1);
  X.F0 = k3 * f0;
  X.F1 = k1 * f1;
  X.D0 = k1 * d0;
  X.D1 = k1 * d1;
  return X;
}

// The same values for the (n, m) = (3, 2) power law with the constant
// factors folded on the host (LineK): the Laplacian is left unscaled and
// 1/ds^2 moves into D0, so faces see the same products.
template <class LP, class Acc>
__device__ __forceinline__ CellS<LP> cell_pl32(const LineK<LP>& L, Acc U) {
  CellS<LP> X;
  const LP uc = U(0, 0);
  X.u = uc;
  X.lap = ((U(0, 1) - uc) + (U(0, -1) - uc)) + ((U(1, 0) - uc) + (U(-1, 0) - uc));
  const LP s = rcp(uc), h2 = uc * uc;
  // F0 rounded as a product of its own (never fused into the face sums
  // F0_p + F0_q) and F1 as one written-out fma: every instantiation of the
  // sweeps then rounds the band alike
  X.F0 = mul_rn(L.pF0, h2 * uc);
  X.F1 = fma(-L.pF1b, s, L.pF1a);
  X.D0 = L.pD0 * h2;
  X.D1 = L.pD1 * (s * s);
  return X;
}

template <class LP>
__device__ __forceinline__ void face_scaled(const CellS<LP>& P, const CellS<LP>& Q, bool pl, bool qr,
                                            LP dF[4]) {
  const LP dl = Q.lap - P.lap, du = Q.u - P.u;
  const LP c3 = P.F0 + Q.F0, Bd = P.F1 + Q.F1;
  // one fused form, written out, so that every instantiation of the sweeps
  // rounds these alike (a * b + c * d may otherwise fuse either product)
  const LP tp = fma(P.D0, dl, P.D1 * du), tq = fma(Q.D0, dl, Q.D1 * du);
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

// Band rows of the cells ia .. ib-1 (at most G) of one line, built in
// registers straight from the staged film tile: the scaled film values of the
// G + 2 cells ia-1 .. ia+G, the G + 1 faces between them, and each row from
// the derivatives of its two face fluxes (a..e multiply x_{i-2}..x_{i+2}).
// A(s, dr, dc) is the film at line cell ia + s offset by (dr, dc) in the grid.
// EDGE: the group may reach a wall, where the outer face of an end cell
// vanishes and faces next to a wall lose their outer stencil weight; without
// EDGE (ia >= 2 and ia + G + 1 < n) every face is interior.  PL32 selects
// the folded (n, m) = (3, 2) power law.  OUT(s, a, b, c, d, e) receives the
// row of cell ia + s.
template <class LP, int G, bool EDGE, bool PL32, class Acc, class Out>
__device__ __forceinline__ void band_rows(const LineK<LP>& L, Acc A, int ia, int ib, int n, Out out) {
  CellS<LP> C[G + 2];
#pragma unroll
  for (int s = -1; s <= G; ++s) {
    auto U = [&](int dr, int dc) { return A(s, dr, dc); };
    if constexpr (PL32)
      C[s + 1] = cell_pl32<LP>(L, U);
    else
      C[s + 1] = cell_scaled<LP>(L.ml, L.inv_ds2, L.k3, L.k1, U);
  }
  LP F[G + 1][4];
#pragma unroll
  for (int f = 0; f <= G; ++f) {  // face between cells ia + f - 1 and ia + f
    if (EDGE) {
      const int q = ia + f - 1;
      face_scaled(C[f], C[f + 1], q > 0, q + 2 < n, F[f]);
      if (!(q >= 0 && q + 1 < n))
        for (int k = 0; k < 4; ++k) F[f][k] = LP(0);
    } else {
      face_scaled(C[f], C[f + 1], true, true, F[f]);
    }
  }
#pragma unroll
  for (int s = 0; s < G; ++s)
    if (ia + s < ib)
      out(s, -F[s][0], F[s + 1][0] - F[s][1], LP(1) + (F[s + 1][1] - F[s][2]), F[s + 1][2] - F[s][3],
          F[s + 1][3]);
}

// Forward elimination over the n cells of one chunk in the band buffer B
// ([a..e, r][cell][line]), cell 0 first.  The producers store both halves of
// a twisted line in this processing order -- the second half with its band
// reversed (e..a) and its cells from the far end -- so one code path serves
// both solver warps.  The factors go to Q[f * L * 32 + s * 32] (this lane's
// column of the chunk's factor slab).  A zero or non-finite pivot sets bad.
// The loop is unrolled so that band loads run ahead of the recurrence.
template <class LP, int L>
__device__ __forceinline__ void lu_chunk(LUState<LP>& lu, const LP* B, int lane, int n, LP* Q, int& bad) {
  LP chk = LP(0);
  auto one = [&](int s) {
    const int k = s * 32 + lane;
    LP g, dl, z;
    lu.step(B[k], B[L * 32 + k], B[2 * L * 32 + k], B[3 * L * 32 + k], B[4 * L * 32 + k], B[5 * L * 32 + k],
            g, dl, z, chk);
    Q[s * 32] = g;
    Q[L * 32 + s * 32] = dl;
    Q[2 * L * 32 + s * 32] = z;
  };
  if (n == L) {  // a whole chunk: every address is an immediate offset
#pragma unroll
    for (int s = 0; s < L; ++s) one(s);
  } else {
#pragma unroll 8
    for (int s = 0; s < n; ++s) one(s);
  }
  if (!(chk == chk)) bad = 1;
}

// Factor scratch of a sweep: for every block of 32 lines, line half and
// chunk, one slab [g, d, z][cell][line] of 3 * L * 32 values, cells in the
// solver's processing order; the backward pass stages a slab with one
// contiguous copy.
template <int L> __host__ __device__ inline int chunks_per_half(int n) {
  const int m = split_point<L>(n);
  const int a = (m + L - 1) / L, b = m < n ? (n - m + L - 1) / L : 0;
  return a > b ? a : b;
}
template <int L> __host__ __device__ inline size_t fac_slab(int blk, int h, int q, int nch) {
  return (((size_t)blk * 2 + h) * nch + q) * (size_t)(3 * L * 32);
}

// Back substitution x = z - g x' - d x'' over the n cells of one chunk in
// processing order s = 0..n-1 (outward from the seam).  F(f, s) reads factor
// f (g, d, z) of cell s; cells with IS_SEAM(s) take the seam solution XS(s);
// PUT(s, x) stores x.  Chunks without seam cells run unrolled.
template <class LP, int L, class Fac, class SeamF, class XsF, class Put>
__device__ __forceinline__ void bs_chunk(LP& x1, LP& x2, int n, bool any_seam, Fac F, SeamF is_seam,
                                         XsF xs, Put put) {
  auto one = [&](int s, bool chk) {
    const LP x = (chk && is_seam(s)) ? xs(s) : F(2, s) - F(0, s) * x1 - F(1, s) * x2;
    x2 = x1;
    x1 = x;
    put(s, x);
  };
  if (!any_seam && n == L) {
#pragma unroll
    for (int s = 0; s < L; ++s) one(s, false);
  } else if (!any_seam) {
#pragma unroll 8
    for (int s = 0; s < n; ++s) one(s, false);
  } else {
    for (int s = 0; s < n; ++s) one(s, true);
  }
}

// ---------------------------------------------------------------------------
// y sweep.  Block: 32 columns i0..i0+31.  Warp 0 / 1 solve the top / bottom
// halves; warps 2..9 produce.  Producer thread p builds the band rows of
// half p >> 7, column p & 31 and the row group (p >> 5) & 3 (kG rows of a
// kRY-row chunk).  Film tiles are staged from the LP film: the FP32 copy that
// k_rhs wrote in FP32-bulk, u_k itself in FP64.

template <class LP> struct YFwd {
  LP ut[2][2][kRY + 4][40];      // LP film tiles (rows r0-2.., cols i0-4..i0+35)
  LP wt[2][2][kRY][32];          // right sides w
  LP band[2][2][6][kRY][32];     // [stage][half][a..e, r][row][col]
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

// DEV (the ensemble graphs): the step's band constants *Ld and the
// iterates {u_k, u_k+1} = uio[0], uio[1] come from device memory.
template <class Mode, bool DEV = false>
__global__ void __launch_bounds__(kSweepThreads, Mode::kSweepBlocks)
    k_ysweep(ModelK M, LineK<typename Mode::LP> Lp, const double* __restrict__ up,
             const typename Mode::LP* __restrict__ ul, const typename Mode::LP* __restrict__ w,
             typename Mode::LP* __restrict__ fac, double* __restrict__ unp, double* __restrict__ vout,
             PartY* __restrict__ part, const LineK<typename Mode::LP>* __restrict__ Ld = nullptr,
             const double* const* __restrict__ uio = nullptr) {
  typedef typename Mode::LP LP;
  const LineK<LP>& L = DEV ? *Ld : Lp;
  const double* __restrict__ u = DEV ? uio[0] : up;
  double* __restrict__ unew = DEV ? const_cast<double*>(uio[1]) : unp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  YSmem<LP>& S = *reinterpret_cast<YSmem<LP>*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool solver = warp < 2;
  const int p = threadIdx.x - 64;  // producer index (valid when !solver)
  const int nx = M.nx, ny = M.ny;
  const int i0 = blockIdx.x * 32;
  const int m = split_point<kRY>(ny);
  const bool twisted = m < ny;
  // chunks per half (a runtime-indexed array would live in local memory)
  const int nch0 = (m + kRY - 1) / kRY, nch1 = twisted ? (ny - m + kRY - 1) / kRY : 0;
  const int nch = max(nch0, nch1);
  auto nchh = [&](int h) { return h ? nch1 : nch0; };
  auto r0_of = [&](int h, int q) { return h == 0 ? q * kRY : max(m, ny - (q + 1) * kRY); };
  auto r1_of = [&](int h, int q) { return h == 0 ? min(m, (q + 1) * kRY) : ny - q * kRY; };
  int pivot_bad = 0;

  // ---------------- producer helpers ----------------
  // issue the film and w tiles of chunk q of both halves into ring slot q & 1
  auto issue_fwd = [&](int q) {
    const int slot = q & 1;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (q >= nchh(h)) continue;
      const int r0 = r0_of(h, q), r1 = r1_of(h, q);
      copy_tile<LP, kRY + 4, 40, 40>(&S.s.f.ut[slot][h][0][0], ul, r0 - 2, i0 - 4, ny, nx, p);
      copy_rows<LP, kRY, 32, 32>(&S.s.f.wt[slot][h][0][0], w, r0, i0, r1 - r0, nx, p);
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
        // band rows: thread p builds rows ja..jb-1 of column c of half h
        {
          const int h = p >> 7, g = (p >> 5) & 3, c = p & 31;
          if (t < nchh(h) && i0 + c < nx) {
            const int r0 = r0_of(h, t), r1 = r1_of(h, t);
            const int ja = r0 + kG * g, jb = min(r1, ja + kG);
            if (ja < jb) {
              // band in the solver's processing order (see lu_chunk)
              // row of cell ja + s at P + s * ks; the second half's band
              // reversed (e..a) by swapping values, so that every store is
              // an immediate offset from one pointer
              LP* P = &S.s.f.band[t & 1][h][0][0][0] + (h ? r1 - 1 - ja : ja - r0) * 32 + c;
              const int ks = h ? -32 : 32;
              const LP* W = &S.s.f.wt[slot][h][ja - r0][c];
              const LP* T = &S.s.f.ut[slot][h][ja - r0 + 2][c + 4];  // cell ja in the tile
              auto A = [&](int s, int dr, int dc) { return T[(s + dr) * 40 + dc]; };
              auto out = [&](int s, LP a, LP b, LP cc, LP d, LP e) {
                LP* q = P + s * ks;
                q[0] = h ? e : a;
                q[kRY * 32] = h ? d : b;
                q[2 * kRY * 32] = cc;
                q[3 * kRY * 32] = h ? b : d;
                q[4 * kRY * 32] = h ? a : e;
                q[5 * kRY * 32] = W[s * 32];
              };
              const bool edge = !(ja >= 2 && ja + kG + 1 < ny);
              if (!L.ml.pl32)  // general exponents or the linear model
                band_rows<LP, kG, true, false>(L, A, ja, jb, ny, out);
              else if (!edge)
                band_rows<LP, kG, false, true>(L, A, ja, jb, ny, out);
              else
                band_rows<LP, kG, true, true>(L, A, ja, jb, ny, out);
            }
          }
        }
      }
    } else if (t >= 1) {
      const int q = t - 1, h = warp;
      if (q < nchh(h) && i0 + lane < nx) {
        const int r0 = r0_of(h, q), r1 = r1_of(h, q);
        const LP* B = &S.s.f.band[q & 1][h][0][0][0];
        lu_chunk<LP, kRY>(lu, B, lane, r1 - r0, fac + fac_slab<kRY>(blockIdx.x, h, q, nch) + lane, pivot_bad);
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
  // chunk order: b-th backward chunk of half h is chunk nchh(h)-1-b.
  auto issue_bwd_f = [&](int bq) {  // factor tiles of backward chunk bq
    const int slot = bq % 3;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = nchh(h) - 1 - bq;
      if (q < 0) continue;
      copy_span<LP, 3 * kRY * 32>(&S.s.b.ft[slot][h][0][0][0], fac + fac_slab<kRY>(blockIdx.x, h, q, nch),
                                  3 * kRY * 32, p);
    }
  };
  auto issue_bwd_u = [&](int bq) {  // u_k tiles of backward chunk bq
    const int slot = bq % 3;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = nchh(h) - 1 - bq;
      if (q < 0) continue;
      const int r0 = r0_of(h, q), r1 = r1_of(h, q);
      copy_rows<double, kRY, 32, 32>(&S.s.b.ukt[slot][h][0][0], u, r0, i0, r1 - r0, nx, p);
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
        const int h = warp, q = nchh(h) - 1 - t;
        if (q >= 0 && i0 + lane < nx) {
          const int r0 = r0_of(h, q), r1 = r1_of(h, q);
          const int slot = t % 3;
          LP* X = &S.s.b.xb[t & 1][h][0][0];
          // processed cell s is chunk row n-1-s (top half, upward) or s; its
          // factors are slab cell n-1-s (the forward pass ran the other way)
          const int n = r1 - r0, rb = h ? 0 : n - 1, rs = h ? 1 : -1;
          auto F = [&](int f, int s) { return S.s.b.ft[slot][h][f][n - 1 - s][lane]; };
          auto xs = [&](int s) { return S.xs[lane][r0 + rb + rs * s - (m - 2)]; };
          auto put = [&](int s, LP x) { X[(rb + rs * s) * 32 + lane] = x; };
          auto is_seam = [&](int s) {
            const int j = r0 + rb + rs * s;
            return twisted && (h ? j <= m + 1 : j >= m - 2);
          };
          bs_chunk<LP, kRY>(x1, x2, n, twisted && (h ? r0 <= m + 1 : r1 > m - 2), F, is_seam, xs, put);
        }
      }
    } else {
      // finish backward chunk t-1: update, store, reduce
      if (t >= 1) {
        const int bq = t - 1, slot = bq % 3;
        // the 2 * kRY * 32 cells of both halves over the producers: thread p
        // takes column p & 31 and rows rg, rg + 8, rg + 16 of each half, so
        // the row and address arithmetic is done once per half
        const int c = p & 31, rg = p >> 5, col = i0 + c;
        static_assert(kRY % 8 == 0 && kNP == 256, "eight row groups of 32 columns");
        if (col < nx) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int q = nchh(h) - 1 - bq;
            if (q < 0) continue;
            const int r0 = r0_of(h, q), nr = r1_of(h, q) - r0;
            const size_t base = (size_t)(r0 + rg) * nx + col, step8 = (size_t)8 * nx;
#pragma unroll
            for (int i = 0; i < kRY / 8; ++i) {
              const int r = rg + 8 * i;
              if (r >= nr) break;
              const LP x = S.s.b.xb[bq & 1][h][r][c];
              const double uk = S.s.b.ukt[slot][h][r][c];
              // one native FP64 add per cell, correctly rounded (fewer
              // instructions than the integer add of tf_numeric.cuh,
              // measured); the float widened exactly off the FP64 pipe
              const double un = uk + widen_exact(x);
              const size_t idx = base + i * step8;
              unew[idx] = un;
              if (vout) vout[idx] = to_f64(x);
              LP ru = rel_update(x, uk);
              if (!(ru <= err)) err = ru;
              if (!positive_finite_bits(un)) nonfinite = 1;
            }
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
    pp.mass.lo = pp.mass.hi = 0ull;
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
      mass_add(a.mass, b.mass);
      a.nonfinite |= b.nonfinite;
      a.pivot |= b.pivot;
    }
    part[blockIdx.x] = a;
  }
}

// ---------------------------------------------------------------------------
// x sweep.  Block: 32 rows j0..j0+31.  Warp 0 / 1 solve the left / right
// halves of the rows (lane = row); warps 2..9 produce.  Producer thread p
// builds the band rows of half p >> 7, row p & 31 and the column group
// (p >> 5) & 3 (kG columns of a kCX-column chunk).  Factor scratch: one slab
// per block, half and chunk (fac_slab).

template <class LP> struct XFwd {
  LP ut[2][2][34][kCX + 5];      // LP film tiles (rows j0-1.., cols c0-2..c0+kCX+1)
  LP rt[2][2][32][kCX + 1];      // right sides
  LP band[2][2][6][kCX][32];     // [stage][half][a..e, r][col][row]
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

// DEV (the ensemble graphs): the step's band constants *Ld come from device
// memory.
template <class Mode, bool DEV = false>
__global__ void __launch_bounds__(kSweepThreads, Mode::kSweepBlocks)
    k_xsweep(ModelK M, LineK<typename Mode::LP> Lp, const typename Mode::LP* __restrict__ ul,
             typename Mode::LP* __restrict__ rw, typename Mode::LP* __restrict__ fac,
             PartX* __restrict__ part, const LineK<typename Mode::LP>* __restrict__ Ld = nullptr) {
  typedef typename Mode::LP LP;
  const LineK<LP>& L = DEV ? *Ld : Lp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  XSmem<LP>& S = *reinterpret_cast<XSmem<LP>*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool solver = warp < 2;
  const int p = threadIdx.x - 64;
  const int nx = M.nx, ny = M.ny;
  const int j0 = blockIdx.x * 32;
  const int m = split_point<kCX>(nx);
  const bool twisted = m < nx;
  const int nch0 = (m + kCX - 1) / kCX, nch1 = twisted ? (nx - m + kCX - 1) / kCX : 0;
  const int nch = max(nch0, nch1);
  auto nchh = [&](int h) { return h ? nch1 : nch0; };
  auto c0_of = [&](int h, int q) { return h == 0 ? q * kCX : max(m, nx - (q + 1) * kCX); };
  auto c1_of = [&](int h, int q) { return h == 0 ? min(m, (q + 1) * kCX) : nx - q * kCX; };
  int pivot_bad = 0;

  auto issue_fwd = [&](int q) {
    const int slot = q & 1;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (q >= nchh(h)) continue;
      const int c0 = c0_of(h, q), c1 = c1_of(h, q);
      copy_tile<LP, 34, kCX + 4, kCX + 5>(&S.s.f.ut[slot][h][0][0], ul, j0 - 1, c0 - 2, ny, nx, p);
#pragma unroll 1
      copy_rows_elem<LP, 32, kCX, kCX + 1>(&S.s.f.rt[slot][h][0][0], rw + (size_t)j0 * nx + c0, nx,
                                           min(32, ny - j0), c1 - c0, p);
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
        // band rows: thread p builds rows ia..ib-1 of row r of half h
        {
          const int h = p >> 7, g = (p >> 5) & 3, r = p & 31;
          if (t < nchh(h) && j0 + r < ny) {
            const int c0 = c0_of(h, t), c1 = c1_of(h, t);
            const int ia = c0 + kG * g, ib = min(c1, ia + kG);
            if (ia < ib) {
              // band in the solver's processing order (see lu_chunk)
              // row of cell ia + s at P + s * ks, stored as in the y sweep
              LP* P = &S.s.f.band[t & 1][h][0][0][0] + (h ? c1 - 1 - ia : ia - c0) * 32 + r;
              const int ks = h ? -32 : 32;
              const LP* R = &S.s.f.rt[slot][h][r][ia - c0];
              const LP* T = &S.s.f.ut[slot][h][r + 1][ia - c0 + 2];  // cell ia in the tile
              auto A = [&](int s, int dr, int dc) { return T[dr * (kCX + 5) + s + dc]; };
              auto out = [&](int s, LP a, LP b, LP c, LP d, LP e) {
                LP* q = P + s * ks;
                q[0] = h ? e : a;
                q[kCX * 32] = h ? d : b;
                q[2 * kCX * 32] = c;
                q[3 * kCX * 32] = h ? b : d;
                q[4 * kCX * 32] = h ? a : e;
                q[5 * kCX * 32] = R[s];
              };
              const bool edge = !(ia >= 2 && ia + kG + 1 < nx);
              if (!L.ml.pl32)  // general exponents or the linear model
                band_rows<LP, kG, true, false>(L, A, ia, ib, nx, out);
              else if (!edge)
                band_rows<LP, kG, false, true>(L, A, ia, ib, nx, out);
              else
                band_rows<LP, kG, true, true>(L, A, ia, ib, nx, out);
            }
          }
        }
      }
    } else if (t >= 1) {
      const int q = t - 1, h = warp;
      if (q < nchh(h) && j0 + lane < ny) {
        const int c0 = c0_of(h, q), c1 = c1_of(h, q);
        const LP* B = &S.s.f.band[q & 1][h][0][0][0];
        lu_chunk<LP, kCX>(lu, B, lane, c1 - c0, fac + fac_slab<kCX>(blockIdx.x, h, q, nch) + lane, pivot_bad);
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
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = nchh(h) - 1 - bq;
      if (q < 0) continue;
      copy_span<LP, 3 * kCX * 32>(&S.s.b.ft[slot][h][0][0][0], fac + fac_slab<kCX>(blockIdx.x, h, q, nch),
                                  3 * kCX * 32, p);
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
        const int h = warp, q = nchh(h) - 1 - t;
        if (q >= 0 && j0 + lane < ny) {
          const int c0 = c0_of(h, q), c1 = c1_of(h, q);
          const int slot = t % 3;
          // processed cell s is chunk column n-1-s (left half, leftward) or s;
          // its factors are slab cell n-1-s
          const int n = c1 - c0, cb = h ? 0 : n - 1, cs = h ? 1 : -1;
          auto F = [&](int f, int s) { return S.s.b.ft[slot][h][f][n - 1 - s][lane]; };
          auto xs = [&](int s) { return S.xs[lane][c0 + cb + cs * s - (m - 2)]; };
          auto put = [&](int s, LP x) { S.s.b.xb[t & 1][h][cb + cs * s][lane] = x; };
          auto is_seam = [&](int s) {
            const int i = c0 + cb + cs * s;
            return twisted && (h ? i <= m + 1 : i >= m - 2);
          };
          bs_chunk<LP, kCX>(x1, x2, n, twisted && (h ? c0 <= m + 1 : c1 > m - 2), F, is_seam, xs, put);
        }
      }
    } else {
      if (t >= 1) {  // store w of backward chunk t-1, coalesced along rows
        const int bq = t - 1;
        static_assert((32 * kCX) % kNP == 0, "whole copy rounds");
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int q = nchh(h) - 1 - bq;
          if (q < 0) continue;
          const int c0 = c0_of(h, q), nc = c1_of(h, q) - c0;
          LP* dst = rw + (size_t)j0 * nx + c0;
          const LP* X = &S.s.b.xb[bq & 1][h][0][0];
#pragma unroll
          for (int i = 0; i < 32 * kCX / kNP; ++i) {
            const int k = p + i * kNP, r = k / kCX, c = k - r * kCX;
            if (j0 + r < ny && c < nc) dst[(size_t)r * nx + c] = X[c * 33 + r];
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
