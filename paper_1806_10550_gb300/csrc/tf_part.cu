// tf_part.cu -- launches of the partitioned line solves (tf_partition.cuh)
// for the FP32-bulk path of a context.
#include "tf_internal.h"
#include "tf_partition.cuh"

namespace tf {
namespace part {

// ---------------------------------------------------------------------------
// x phase 1: tile of kRX rows x x segment blockIdx.x (the block exists only
// for grids with more than one x segment whose segments are not the
// residual kernel's tiles).

struct X1Smem {
  float film[(kRX + 2) * (kLX + 9)];   // rows j0-1.., cols c0-2 .. c1+3 (odd pitch kLX + 9)
  float rt[kRX * (kLX + 1)];           // right side [row][cell]
  float band[(kLX + 2) * 5 * kRX];     // cells c0 .. c1+1
  float X[2][kRX][10];
};

__global__ void __launch_bounds__(kT, 3)
    k_part_x1(ModelK M, LineK<float> L, const float* __restrict__ ul, const float* __restrict__ r,
              float* __restrict__ rec, Acc* __restrict__ acc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  X1Smem& S = *reinterpret_cast<X1Smem*>(smem_raw);
  constexpr int FP = kLX + 9, RP = kLX + 1;
  const int nx = M.nx, ny = M.ny, nS = seg_count<kLX>(nx);
  const int k = blockIdx.x, j0 = blockIdx.y * kRX;
  const int c0 = seg_start<kLX>(k, nx), c1 = seg_end<kLX>(k, nx), len = c1 - c0;
  const bool next = k + 1 < nS;
  const int ncell = len + (next ? 2 : 0);
  const int nrow = min(kRX, ny - j0);
  load_tile_f32<kRX + 2, kLX + 8, FP, kT>(S.film, ul, j0 - 1, nrow + 2, c0 - 2, ncell + 4, ny, nx);
  load_tile_f32<kRX, kLX, RP, kT>(S.rt, r, j0, nrow, c0, len, ny, nx);
  __syncthreads();
  const LineK2 K = pack_consts(L);
  auto film = [&](int pair, int cell, int dr, int dc) {
    const float* f = S.film + (2 * pair + 1 + dr) * FP + (cell - c0 + 2 + dc);
    return make_float2(f[0], f[FP]);
  };
  build_band<kRX, kT>(K, S.band, nrow, c0, ncell, nx, film);
  __syncthreads();
  int bad = 0;
  phase1<kRX>(S.band, S.X, nrow, k, nS, len, [&](int line, int cell) { return S.rt[line * RP + cell]; }, rec,
              (size_t)ny, (size_t)j0, bad);
  flag_bad(acc, bad);
}

// ---------------------------------------------------------------------------
// Phase 2: the reduced block-tridiagonal systems of 32 lines per block, one
// line per lane.  Row s (s = 1..N, N = S - 1) reads L_s x_{s-1} + D_s x_s +
// U_s x_{s+1} = r_s with D_s = Dp + Dm, r_s = rp + rm, U_s (own record),
// L_s = Lw (next record of segment s - 1).  Warp 0 eliminates rows 1..m
// top-down (W_s = D_s - L_s W_{s-1}^-1 U_{s-1}), warp 1 rows N..m+1
// bottom-up (V_s = D_s - U_s V_{s+1}^-1 L_{s+1}); the 4 x 4 system of rows m
// and m + 1 gives x_m, x_{m+1} (partial pivoting), and both warps
// substitute back outward.  Block LU without pivoting elsewhere, as in the
// line solves.  Records stream through shared memory in chunks of kRCH
// rows, two chunks in flight; each row's inverse pivot block and reduced
// right side overwrite its values 14..19 (already consumed).  xs receives
// [s - 1][2][nlines].

constexpr int kRCH = 8;  // record rows per staged chunk

struct RedSmem {
  float buf[2][2][kRCH][kRec][32];  // [warp][slot][row][value][lane]
  float seam[6][32];
};

__device__ __forceinline__ M2 inv2(const M2& D, int& bad) {
  const float det = D.a * D.d - D.b * D.c;
  const float id = rcp(det);  // the MUFU reciprocal: FP32 solves
  if (!(det != 0.f) || !(id - id == 0.f)) bad = 1;
  return mk2(D.d * id, -D.b * id, -D.c * id, D.a * id);
}

__global__ void __launch_bounds__(64)
    k_part_red(float* __restrict__ rec, int nS, int nlines, float* __restrict__ xs, Acc* __restrict__ acc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RedSmem& S = *reinterpret_cast<RedSmem*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int line = blockIdx.x * 32 + lane;
  const bool valid = line < nlines;
  const size_t NL = (size_t)nlines;
  const int N = nS - 1, m = N >= 2 ? N / 2 : N;
  const int nrows = warp == 0 ? m : N - m;  // rows this warp eliminates
  auto row_of = [&](int t) { return warp == 0 ? 1 + t : N - t; };
  const int nch = (nrows + kRCH - 1) / kRCH;
  auto stage = [&](int c) {
    if (c < nch && valid)
      for (int j = 0; j < kRCH; ++j) {
        const int t = c * kRCH + j;
        if (t >= nrows) break;
        const float* src = rec + (size_t)(row_of(t) - 1) * kRec * NL + line;
#pragma unroll
        for (int q = 0; q < kRec; ++q) cpT(&S.buf[warp][c & 1][j][q][lane], src + q * NL);
      }
    __pipeline_commit();
  };
  int bad = 0;
  M2 W = mk2(0.f, 0.f, 0.f, 0.f), Wi = W, Cprev = W;
  float g0 = 0.f, g1 = 0.f;
  stage(0);
  stage(1);
  for (int c = 0; c < nch; ++c) {
    __pipeline_wait_prior(1);
    __syncwarp();
    for (int j = 0; j < kRCH; ++j) {
      const int t = c * kRCH + j;
      if (t >= nrows) break;
      const float* v = &S.buf[warp][c & 1][j][0][lane];
      auto V = [&](int q) { return v[q * 32]; };
      M2 D = mk2(V(0) + V(14), V(1) + V(15), V(2) + V(16), V(3) + V(17));
      float h0 = V(8) + V(18), h1 = V(9) + V(19);
      // top: L_s couples to the row before; bottom: U_s to the row after
      const M2 Cin = warp == 0 ? mk2(V(10), V(11), V(12), V(13)) : mk2(V(4), V(5), V(6), V(7));
      if (t > 0) {
        const M2 Lam = mul2(Cin, Wi);
        D = sub2(D, mul2(Lam, Cprev));
        float l0, l1;
        mv2(Lam, g0, g1, l0, l1);
        h0 -= l0;
        h1 -= l1;
      }
      W = D;
      Wi = inv2(D, bad);
      g0 = h0;
      g1 = h1;
      // the coupling the next row of this warp's order eliminates through
      Cprev = warp == 0 ? mk2(V(4), V(5), V(6), V(7)) : mk2(V(10), V(11), V(12), V(13));
      if (valid) {
        float* o = rec + ((size_t)(row_of(t) - 1) * kRec + 14) * NL + line;
        o[0] = Wi.a;
        o[NL] = Wi.b;
        o[2 * NL] = Wi.c;
        o[3 * NL] = Wi.d;
        o[4 * NL] = g0;
        o[5 * NL] = g1;
      }
    }
    __syncwarp();
    stage(c + 2);
  }
  __pipeline_wait_prior(0);
  // ---- the seam: [[W_m, U_m], [L_{m+1}, V_{m+1}]] [x_m; x_{m+1}] = [g_m; h_{m+1}]
  if (warp == 1 && m < N) {
    S.seam[0][lane] = W.a;
    S.seam[1][lane] = W.b;
    S.seam[2][lane] = W.c;
    S.seam[3][lane] = W.d;
    S.seam[4][lane] = g0;
    S.seam[5][lane] = g1;
  }
  __syncthreads();
  float xm0 = 0.f, xm1 = 0.f;
  if (warp == 0 && valid) {
    if (m < N) {
      const float* um = rec + ((size_t)(m - 1) * kRec + 4) * NL + line;
      const float* ln = rec + ((size_t)m * kRec + 10) * NL + line;
      float A[4][4] = {{W.a, W.b, __ldcg(um), __ldcg(um + NL)},
                       {W.c, W.d, __ldcg(um + 2 * NL), __ldcg(um + 3 * NL)},
                       {__ldcg(ln), __ldcg(ln + NL), S.seam[0][lane], S.seam[1][lane]},
                       {__ldcg(ln + 2 * NL), __ldcg(ln + 3 * NL), S.seam[2][lane], S.seam[3][lane]}};
      float b[4] = {g0, g1, S.seam[4][lane], S.seam[5][lane]}, x[4];
      if (!solve4(A, b, x)) bad = 1;
      xm0 = x[0];
      xm1 = x[1];
      S.seam[0][lane] = x[2];
      S.seam[1][lane] = x[3];
    } else {
      mv2(Wi, g0, g1, xm0, xm1);  // N = 1: the one row
    }
  }
  __syncthreads();
  // ---- back substitution outward, 4 rows of values read ahead
  if (valid) {
    auto put = [&](int s, float a, float b) {
      xs[(size_t)(s - 1) * 2 * NL + line] = a;
      xs[((size_t)(s - 1) * 2 + 1) * NL + line] = b;
    };
    // top: x_s = W_s^-1 (g_s - U_s x_{s+1}), s = m-1..1;
    // bottom: x_s = V_s^-1 (h_s - L_s x_{s-1}), s = m+2..N
    const int s0 = warp == 0 ? m : m + 1, ds = warp == 0 ? -1 : 1, cq = warp == 0 ? 4 : 10;
    float x0 = warp == 0 ? xm0 : S.seam[0][lane], x1 = warp == 0 ? xm1 : S.seam[1][lane];
    if (warp == 0 || m < N) {
      put(s0, x0, x1);
      const int nb = warp == 0 ? m - 1 : N - m - 1;
      for (int b = 0; b < nb; ++b) {
        const int s = s0 + ds * (b + 1);
        const float* r = rec + (size_t)(s - 1) * kRec * NL + line;
        const M2 Cm = mk2(__ldcg(r + cq * NL), __ldcg(r + (cq + 1) * NL), __ldcg(r + (cq + 2) * NL),
                          __ldcg(r + (cq + 3) * NL));
        const M2 Wm = mk2(__ldcg(r + 14 * NL), __ldcg(r + 15 * NL), __ldcg(r + 16 * NL), __ldcg(r + 17 * NL));
        const float e0 = __ldcg(r + 18 * NL), e1 = __ldcg(r + 19 * NL);
        float u0, u1;
        mv2(Cm, x0, x1, u0, u1);
        mv2(Wm, e0 - u0, e1 - u1, x0, x1);
        put(s, x0, x1);
      }
    }
  }
  flag_bad(acc, bad && valid);  // lanes past the last line eliminate garbage
}

// ---------------------------------------------------------------------------
// x phase 3 + y phase 1: tile = y segment blockIdx.y x x segment blockIdx.x.

struct XYSmem {
  float film[(kLY + 6) * (kLX + 5)];   // rows r0-2 .. r1+3, cols c0-2 .. c1+1 (odd pitch kLX + 5)
  float wt[kLY * (kLX + 1)];           // right side r, then w, [row][col]
  // x band [cell < kLX][5][row < kLY], then y band [cell < kLY + 2][5][col < kLX]
  float band[(kLX * kLY > (kLY + 2) * kLX ? kLX * kLY : (kLY + 2) * kLX) * 5];
  Seam2<kLY> seam;
  float xsl[kLY][2], xsr[kLY][2];
  float X[2][kLX][10];
};

__global__ void __launch_bounds__(kT, 3)
    k_part_xy(ModelK M, LineK<float> L, const float* __restrict__ ul, float* __restrict__ rw,
              const float* __restrict__ xsx, float* __restrict__ recy, Acc* __restrict__ acc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  XYSmem& S = *reinterpret_cast<XYSmem*>(smem_raw);
  constexpr int FP = kLX + 5, WP = kLX + 1;
  const int nx = M.nx, ny = M.ny;
  const int nSx = seg_count<kLX>(nx), nSy = seg_count<kLY>(ny);
  const int kx = blockIdx.x, ky = blockIdx.y;
  const int c0 = seg_start<kLX>(kx, nx), c1 = seg_end<kLX>(kx, nx), nc = c1 - c0;
  const int r0 = seg_start<kLY>(ky, ny), r1 = seg_end<kLY>(ky, ny), nr = r1 - r0;
  const bool nexty = ky + 1 < nSy;
  const int nrowy = nr + (nexty ? 2 : 0);  // y band rows: segment + next separator
  load_tile_f32<kLY + 6, kLX + 4, FP, kT>(S.film, ul, r0 - 2, nrowy + 4, c0 - 2, nc + 4, ny, nx);
  load_tile_f32<kLY, kLX, WP, kT>(S.wt, rw, r0, nr, c0, nc, ny, nx);
  for (int q = threadIdx.x; q < 2 * nr; q += kT) {
    const int row = q >> 1, e = q & 1;
    S.xsl[row][e] = kx > 0 ? xsx[((size_t)(kx - 1) * 2 + e) * ny + r0 + row] : 0.f;
    S.xsr[row][e] = kx + 1 < nSx ? xsx[((size_t)kx * 2 + e) * ny + r0 + row] : 0.f;
  }
  __syncthreads();
  const LineK2 K = pack_consts(L);
  // ---- x band of the tile's rows, cells c0 .. c1-1
  {
    auto film = [&](int pair, int cell, int dr, int dc) {
      const float* f = S.film + (2 * pair + 2 + dr) * FP + (cell - c0 + 2 + dc);
      return make_float2(f[0], f[FP]);
    };
    build_band<kLY, kT>(K, S.band, nr, c0, nc, nx, film);
  }
  __syncthreads();
  int bad = 0;
  // ---- x phase 3: interiors of the tile's rows; separators from phase 2
  {
    const int p0 = kx > 0 ? 2 : 0, m = nc - p0;
    const bool right = kx + 1 < nSx;
    auto rhs = [&](int pair, int i) {
      const int cell = p0 + i, l0 = 2 * pair;
      float2 f = make_float2(S.wt[l0 * WP + cell], S.wt[(l0 + 1) * WP + cell]);
      if (kx > 0 && i <= 1) {
        const Row2 B = band_row2<kLY>(S.band, cell, pair, false);
        const float2 s0 = make_float2(S.xsl[l0][0], S.xsl[l0 + 1][0]);
        const float2 s1 = make_float2(S.xsl[l0][1], S.xsl[l0 + 1][1]);
        f = i == 0 ? p_fma(p_neg(B.b), s1, p_fma(p_neg(B.a), s0, f)) : p_fma(p_neg(B.a), s1, f);
      }
      if (right && i >= m - 2) {
        const Row2 B = band_row2<kLY>(S.band, cell, pair, false);
        const float2 s0 = make_float2(S.xsr[l0][0], S.xsr[l0 + 1][0]);
        const float2 s1 = make_float2(S.xsr[l0][1], S.xsr[l0 + 1][1]);
        f = i == m - 2 ? p_fma(p_neg(B.e), s0, f) : p_fma(p_neg(B.e), s1, p_fma(p_neg(B.d), s0, f));
      }
      return f;
    };
    auto put = [&](int pair, int i, float2 x) {
      S.wt[2 * pair * WP + p0 + i] = x.x;
      S.wt[(2 * pair + 1) * WP + p0 + i] = x.y;
    };
    twisted_solve2<kLY>(S.band, S.seam, nr, p0, m, rhs, put, bad);
    if (kx > 0)
      for (int q = threadIdx.x; q < 2 * nr; q += kT) S.wt[(q >> 1) * WP + (q & 1)] = S.xsl[q >> 1][q & 1];
  }
  __syncthreads();
  // ---- store w; y band of the tile's columns, rows r0 .. r1 (+ next separator)
  for (int k = threadIdx.x; k < nr * (kLX / 2); k += kT) {
    const int rr = k / (kLX / 2), cc = 2 * (k - rr * (kLX / 2));
    float* d = rw + (size_t)(r0 + rr) * nx + c0 + cc;
    if (cc + 1 < nc && ((nx | c0) & 1) == 0)
      *reinterpret_cast<float2*>(d) = make_float2(S.wt[rr * WP + cc], S.wt[rr * WP + cc + 1]);
    else {
      if (cc < nc) d[0] = S.wt[rr * WP + cc];
      if (cc + 1 < nc) d[1] = S.wt[rr * WP + cc + 1];
    }
  }
  {
    auto film = [&](int pair, int cell, int dr, int dc) {
      const float* f = S.film + (cell - r0 + 2 + dr) * FP + (2 * pair + 2 + dc);
      return make_float2(f[0], f[1]);
    };
    build_band<kLX, kT>(K, S.band, nc, r0, nrowy, ny, film);
  }
  __syncthreads();
  // ---- y phase 1 (lines = the tile's columns)
  if (nSy > 1)
    phase1<kLX>(S.band, S.X, nc, ky, nSy, nr, [&](int line, int cell) { return S.wt[cell * WP + line]; }, recy,
                (size_t)nx, (size_t)c0, bad);
  flag_bad(acc, bad);
}

// ---------------------------------------------------------------------------
// y phase 3, Newton update and reductions: tile = y segment blockIdx.y x
// kCY columns from blockIdx.x * kCY.

struct YCSmem {
  float film[(kLY + 4) * (kCY + 4)];   // rows r0-2 .. r1+1, cols i0-2 .. i0+kCY+1
  float wt[kLY * (kCY + 2)];           // w, then v, [row][col]
  float band[kLY * 5 * kCY];
  Seam2<kCY> seam;
  float ysl[kCY][2], ysr[kCY][2];
  float red[kT / 32];
  int nf[kT / 32];
};

__global__ void __launch_bounds__(kT, 3)
    k_part_yc(ModelK M, LineK<float> L, const double* __restrict__ u, const float* __restrict__ w,
              const float* __restrict__ xsy, double* __restrict__ unew, double* __restrict__ vout,
              Acc* __restrict__ acc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  YCSmem& S = *reinterpret_cast<YCSmem*>(smem_raw);
  constexpr int FP = kCY + 4, WP = kCY + 2;
  const int nx = M.nx, ny = M.ny, nSy = seg_count<kLY>(ny);
  const int i0 = blockIdx.x * kCY, ky = blockIdx.y;
  const int nc = min(kCY, nx - i0);
  const int r0 = seg_start<kLY>(ky, ny), r1 = seg_end<kLY>(ky, ny), nr = r1 - r0;
  load_tile_f64<kLY + 4, kCY + 4, FP, kT>(S.film, u, r0 - 2, nr + 4, i0 - 2, nc + 4, ny, nx);
  load_tile_f32<kLY, kCY, WP, kT>(S.wt, w, r0, nr, i0, nc, ny, nx);
  for (int q = threadIdx.x; q < 2 * nc; q += kT) {
    const int col = q >> 1, e = q & 1;
    S.ysl[col][e] = ky > 0 ? xsy[((size_t)(ky - 1) * 2 + e) * nx + i0 + col] : 0.f;
    S.ysr[col][e] = ky + 1 < nSy ? xsy[((size_t)ky * 2 + e) * nx + i0 + col] : 0.f;
  }
  __syncthreads();
  {
    const LineK2 K = pack_consts(L);
    auto film = [&](int pair, int cell, int dr, int dc) {
      const float* f = S.film + (cell - r0 + 2 + dr) * FP + (2 * pair + 2 + dc);
      return make_float2(f[0], f[1]);
    };
    build_band<kCY, kT>(K, S.band, nc, r0, nr, ny, film);
  }
  __syncthreads();
  int bad = 0;
  {
    const int p0 = ky > 0 ? 2 : 0, m = nr - p0;
    const bool right = ky + 1 < nSy;
    auto rhs = [&](int pair, int i) {
      const int cell = p0 + i, l0 = 2 * pair;
      float2 f = make_float2(S.wt[cell * WP + l0], S.wt[cell * WP + l0 + 1]);
      if (ky > 0 && i <= 1) {
        const Row2 B = band_row2<kCY>(S.band, cell, pair, false);
        const float2 s0 = make_float2(S.ysl[l0][0], S.ysl[l0 + 1][0]);
        const float2 s1 = make_float2(S.ysl[l0][1], S.ysl[l0 + 1][1]);
        f = i == 0 ? p_fma(p_neg(B.b), s1, p_fma(p_neg(B.a), s0, f)) : p_fma(p_neg(B.a), s1, f);
      }
      if (right && i >= m - 2) {
        const Row2 B = band_row2<kCY>(S.band, cell, pair, false);
        const float2 s0 = make_float2(S.ysr[l0][0], S.ysr[l0 + 1][0]);
        const float2 s1 = make_float2(S.ysr[l0][1], S.ysr[l0 + 1][1]);
        f = i == m - 2 ? p_fma(p_neg(B.e), s0, f) : p_fma(p_neg(B.e), s1, p_fma(p_neg(B.d), s0, f));
      }
      return f;
    };
    auto put = [&](int pair, int i, float2 x) {
      S.wt[(p0 + i) * WP + 2 * pair] = x.x;
      S.wt[(p0 + i) * WP + 2 * pair + 1] = x.y;
    };
    twisted_solve2<kCY>(S.band, S.seam, nc, p0, m, rhs, put, bad);
    if (ky > 0)
      for (int q = threadIdx.x; q < 2 * nc; q += kT) S.wt[(q & 1) * WP + (q >> 1)] = S.ysl[q >> 1][q & 1];
  }
  flag_bad(acc, bad);
  __syncthreads();
  // ---- u_{k+1} = u_k + v (one native FP64 add per cell), max |v/u_k|, positivity
  float err = 0.f;
  int nonfinite = 0;
  for (int k = threadIdx.x; k < nr * kCY; k += kT) {
    const int rr = k / kCY, cc = k - rr * kCY;
    if (cc >= nc) continue;
    const size_t idx = (size_t)(r0 + rr) * nx + i0 + cc;
    const float x = S.wt[rr * WP + cc];
    const double uk = __ldg(u + idx);
    const double un = uk + (double)x;
    unew[idx] = un;
    if (vout) vout[idx] = (double)x;
    const float ru = rel_update(x, uk);
    if (!(ru <= err)) err = ru;
    if (!positive_finite_bits(un)) nonfinite = 1;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const float e2 = __shfl_xor_sync(0xffffffffu, err, o);
    if (!(e2 <= err)) err = e2;
    nonfinite |= __shfl_xor_sync(0xffffffffu, nonfinite, o);
  }
  if ((threadIdx.x & 31) == 0) {
    S.red[threadIdx.x >> 5] = err;
    S.nf[threadIdx.x >> 5] = nonfinite;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float e = S.red[0];
    int n = S.nf[0];
    for (int q = 1; q < kT / 32; ++q) {
      if (!(S.red[q] <= e)) e = S.red[q];
      n |= S.nf[q];
    }
    atomicMax(&acc->err_bits, __float_as_uint(fabsf(e)) | (e == e ? 0u : 0x7fc00000u));
    if (n) atomicOr(&acc->nonfinite, 1);
  }
}

// The iteration's scalars: max |G| from the residual kernel's partials,
// the accumulators of the partitioned kernels (then cleared for the next
// iteration).  One block.
static __global__ void __launch_bounds__(256)
    k_part_finalize(const PartX* __restrict__ px, int nx_part, Acc* __restrict__ acc, Scalars* __restrict__ out) {
  __shared__ double s_g[256];
  __shared__ int s_pv[256];
  const int t = threadIdx.x;
  double g = 0.0;
  int pv = 0;
  for (int k = t; k < nx_part; k += 256) {
    if (!(px[k].gnorm <= g)) g = px[k].gnorm;
    pv |= px[k].pivot;
  }
  s_g[t] = g;
  s_pv[t] = pv;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (t < o) {
      if (!(s_g[t + o] <= s_g[t])) s_g[t] = s_g[t + o];
      s_pv[t] |= s_pv[t + o];
    }
    __syncthreads();
  }
  if (t == 0) {
    Scalars s;
    s.err = (double)__uint_as_float(acc->err_bits);
    s.gnorm = s_g[0];
    s.hmin = INFINITY;
    s.mass.lo = s.mass.hi = 0ull;
    s.nonfinite = acc->nonfinite;
    s.pivot = s_pv[0] | acc->pivot;
    *out = s;
    Acc z;
    z.err_bits = 0u;
    z.nonfinite = 0;
    z.pivot = 0;
    z.pad = 0;
    *acc = z;
  }
}

static_assert(kRec == kRecordValues, "record size shared with the workspace allocation");

int nseg_x(int nx) { return seg_count<kLX>(nx); }
int nseg_y(int ny) { return seg_count<kLY>(ny); }
size_t acc_bytes() { return sizeof(Acc); }

cudaError_t prepare() {
  cudaError_t e;
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  const cudaFuncAttribute C = cudaFuncAttributePreferredSharedMemoryCarveout;
  const int maxc = (int)cudaSharedmemCarveoutMaxShared;
  if ((e = cudaFuncSetAttribute(k_part_x1, A, (int)sizeof(X1Smem)))) return e;
  if ((e = cudaFuncSetAttribute(k_part_xy, A, (int)sizeof(XYSmem)))) return e;
  if ((e = cudaFuncSetAttribute(k_part_yc, A, (int)sizeof(YCSmem)))) return e;
  // a line's records: up to 65536 / 32 - 1 separators of 20 values
  if ((e = cudaFuncSetAttribute(k_part_red, A, (int)sizeof(RedSmem)))) return e;
  if ((e = cudaFuncSetAttribute(k_part_x1, C, maxc))) return e;
  if ((e = cudaFuncSetAttribute(k_part_xy, C, maxc))) return e;
  return cudaFuncSetAttribute(k_part_yc, C, maxc);
}

static LineK<float> consts(const tf_ctx& c, double dt) {
  StepK k;
  k.theta_dt = c.p.theta * dt;
  k.expl_dt = (1.0 - c.p.theta) * dt;
  return line_consts<float>(c.mk, k);
}

cudaError_t xsweep(tf_ctx& c, double dt) {
  const LineK<float> L = consts(c, dt);
  const float* ul = (const float*)c.ulp;
  float* rw = (float*)c.w;
  const int ny = c.mk.ny, nx = c.mk.nx;
  if (c.nsx > 1) {
    k_part_x1<<<dim3(c.nsx, (ny + kRX - 1) / kRX), kT, sizeof(X1Smem), c.stream>>>(c.mk, L, ul, rw, c.recx,
                                                                                 c.acc);
  }
  if (c.nsx > 1)
    k_part_red<<<(ny + 31) / 32, 64, sizeof(RedSmem), c.stream>>>(c.recx, c.nsx, ny, c.xsx, c.acc);
  k_part_xy<<<dim3(c.nsx, c.nsy), kT, sizeof(XYSmem), c.stream>>>(c.mk, L, ul, rw, c.xsx, c.recy, c.acc);
  if (c.nsy > 1)
    k_part_red<<<(nx + 31) / 32, 64, sizeof(RedSmem), c.stream>>>(c.recy, c.nsy, nx, c.xsy, c.acc);
  return cudaGetLastError();
}

cudaError_t ysweep(tf_ctx& c, const double* u_k, double dt, double* u_next, double* v_out) {
  const LineK<float> L = consts(c, dt);
  k_part_yc<<<dim3((c.mk.nx + kCY - 1) / kCY, c.nsy), kT, sizeof(YCSmem), c.stream>>>(
      c.mk, L, u_k, (const float*)c.w, c.xsy, u_next, v_out, c.acc);
  return cudaGetLastError();
}

cudaError_t finalize(tf_ctx& c) {
  k_part_finalize<<<1, 256, 0, c.stream>>>(c.px, c.n_rhs_parts, c.acc, c.dsc);
  return cudaGetLastError();
}

int launches(const tf_ctx& c) { return 2 + (c.nsx > 1 ? 2 : 0) + (c.nsy > 1 ? 1 : 0); }

}  // namespace part
}  // namespace tf
