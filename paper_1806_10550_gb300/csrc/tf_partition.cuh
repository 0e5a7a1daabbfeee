// tf_partition.cuh -- partitioned line solves of the FP32-bulk path.
//
// The pentadiagonal systems (I + theta dt J_x) w = -G on every row and
// (I + theta dt J_y) v = w on every column (eqs. JacobianSystem1-2) are
// solved exactly, as the LU solve of eq. LUFactorization would solve them,
// but each line is cut into segments that are solved independently, with a
// small reduced system per line coupling them (the partition idea the paper
// names as future work in its conclusions):
//
//   line cells 0..n-1, segment k = [B_k, B_{k+1}); separator k (k >= 1) is
//   the two cells B_k, B_k + 1; interior k the rest of segment k.  With the
//   separators known, the interiors decouple (the band reaches two cells).
//
//   phase 1  per segment: two elimination passes over the interior, one from
//            each end, give the 2 x 2 corner blocks of its inverse and its
//            solution for the right side at its first and last two cells;
//            with the band rows of the separators on both sides these make
//            the segment's share of the reduced system (a "record").
//   phase 2  per line: the reduced system on the separators is block
//            tridiagonal with 2 x 2 blocks (the Schur complement of the
//            interiors); block LU without pivoting, then back substitution.
//   phase 3  per segment: the interior's own system with the separators'
//            values moved to the right side, solved by a twisted LU (two
//            threads, meeting in the middle with a 4 x 4 seam solve).
//
// Nothing of a segment is kept between phases but its 20-value record and
// the separators' values: phase 3 rebuilds the band from the film tile.
// Every segment of every line is an independent block of work, so all SMs
// stay busy and no LU factors travel through HBM.
//
// Kernels (FP32 film and solves, the (3, 2) power law or any model through
// band_rows):
//   k_part_x1  x phase 1 on a tile of 32 rows x one x segment (reads the
//              FP32 film and the right side r = -G written by the residual);
//   k_part_red phase 2 of one direction, one thread per line;
//   k_part_xy  x phase 3 on a tile of one y segment x one x segment (writes
//              w), then y phase 1 on the same tile's columns;
//   k_part_yc  y phase 3 on a tile of one y segment x 64 columns, the Newton
//              update u_{k+1} = u_k + v and the iteration's reductions.
#pragma once

#include "tf_line_sweeps.cuh"

namespace tf {
namespace part {

constexpr int kT = 256;    // threads per block
constexpr int kLX = 64;    // x segment length (cells)
constexpr int kLY = 32;    // y segment length (cells)
constexpr int kRX = 32;    // rows per x phase-1 tile
constexpr int kCY = 64;    // columns per y phase-3 tile
constexpr int kRec = 20;   // record values per separator and line
constexpr int kGB = 6;     // band rows one thread builds at a time
static_assert(kCY == kLX, "an xy tile is one x segment wide and holds the y lines of those columns");

// ---------------------------------------------------------------------------
// Segment geometry: S segments of at most L cells; segment k starts at k L,
// except that a last segment that would hold fewer than 4 cells starts at
// n - 4 instead (every interior then has at least 2 cells, so a separator's
// band rows reach only into the adjacent interiors).

template <int L> __host__ __device__ __forceinline__ int seg_count(int n) {
  return n <= L ? 1 : (n + L - 1) / L;
}
template <int L> __host__ __device__ __forceinline__ int seg_start(int k, int n) {
  const int S = seg_count<L>(n);
  return (S > 1 && k == S - 1) ? min(k * L, n - 4) : k * L;
}
template <int L> __host__ __device__ __forceinline__ int seg_end(int k, int n) {
  return k + 1 < seg_count<L>(n) ? seg_start<L>(k + 1, n) : n;
}

// 2 x 2 matrices, row-major [[a, b], [c, d]]
struct M2 {
  float a, b, c, d;
};
__device__ __forceinline__ M2 mk2(float a, float b, float c, float d) {
  M2 m;
  m.a = a;
  m.b = b;
  m.c = c;
  m.d = d;
  return m;
}
__device__ __forceinline__ M2 mul2(const M2& x, const M2& y) {
  return mk2(x.a * y.a + x.b * y.c, x.a * y.b + x.b * y.d, x.c * y.a + x.d * y.c, x.c * y.b + x.d * y.d);
}
__device__ __forceinline__ M2 sub2(const M2& x, const M2& y) {
  return mk2(x.a - y.a, x.b - y.b, x.c - y.c, x.d - y.d);
}
__device__ __forceinline__ void mv2(const M2& x, float u, float v, float& p, float& q) {
  p = x.a * u + x.b * v;
  q = x.c * u + x.d * v;
}

// Band rows in shared memory: band[(cell * 5 + q) * NL + line], q = a..e
// (multiplying x_{i-2}..x_{i+2}).  A row in the orientation of a pass:
// natural, or reversed (the line read backwards: e..a).
struct Row {
  float a, b, c, d, e;
};
template <int NL>
__device__ __forceinline__ Row band_row(const float* band, int cell, int line, bool rev) {
  const float* p = band + cell * 5 * NL + line;
  Row r;
  if (!rev) {
    r.a = p[0];
    r.b = p[NL];
    r.c = p[2 * NL];
    r.d = p[3 * NL];
    r.e = p[4 * NL];
  } else {
    r.e = p[0];
    r.d = p[NL];
    r.c = p[2 * NL];
    r.b = p[3 * NL];
    r.a = p[4 * NL];
  }
  return r;
}

// Build the band rows of cells [ia0, ia0 + ncell) of nl lines into band
// (cell index relative to ia0).  film(line, cell, dr, dc) gives the FP32
// film at line `line`, line cell `cell` (global index along the line),
// offset by dr cells across and dc along the line.  n: line length.
template <int NL, class Film>
__device__ __forceinline__ void build_band(const LineK<float>& L, float* band, int nl, int ia0, int ncell,
                                           int n, Film film) {
  const int ngrp = (ncell + kGB - 1) / kGB;
  for (int task = threadIdx.x; task < ngrp * NL; task += kT) {
    const int line = task % NL, grp = task / NL;
    if (line >= nl) continue;
    const int ia = ia0 + grp * kGB, ib = min(ia0 + ncell, ia + kGB);
    auto A = [&](int s, int dr, int dc) { return film(line, ia + s, dr, dc); };
    float* P = band + (ia - ia0) * 5 * NL + line;
    auto out = [&](int s, float a, float b, float c, float d, float e) {
      float* q = P + s * 5 * NL;
      q[0] = a;
      q[NL] = b;
      q[2 * NL] = c;
      q[3 * NL] = d;
      q[4 * NL] = e;
    };
    const bool edge = !(ia >= 2 && ia + kGB + 1 < n);
    if (!L.ml.pl32)
      band_rows<float, kGB, true, false>(L, A, ia, ib, n, out);
    else if (!edge)
      band_rows<float, kGB, false, true>(L, A, ia, ib, n, out);
    else
      band_rows<float, kGB, true, true>(L, A, ia, ib, n, out);
  }
}

// Phase 1: one elimination pass over an interior of m >= 2 rows, LU without
// pivoting of the interior's own matrix (entries that reach outside it
// dropped), with the right sides f and the unit vectors e_0, e_1.  X
// receives rows m-2 and m-1 (in the pass's orientation) of A^-1 applied to
// [f, e_0, e_1, e_{m-2}, e_{m-1}].  ROW(i) gives row i in the pass's
// orientation; RHS(i) its right side.  A zero or non-finite pivot sets bad.
template <class RowF, class RhsF>
__device__ __forceinline__ void elim_pass(RowF ROW, RhsF RHS, int m, float X[2][5], int& bad) {
  float g1 = 0.f, d1 = 0.f, g2 = 0.f, d2 = 0.f;
  float zf1 = 0.f, zf2 = 0.f, za1 = 0.f, za2 = 0.f, zb1 = 0.f, zb2 = 0.f;
  float gm2 = 0.f, im2 = 0.f, bm1 = 0.f, im1 = 0.f, chk = 0.f;
#pragma unroll 4
  for (int i = 0; i < m; ++i) {
    Row R = ROW(i);
    const float f = RHS(i);
    if (i == 0) R.b = 0.f;
    if (i <= 1) R.a = 0.f;
    if (i + 1 >= m) R.d = 0.f;
    if (i + 2 >= m) R.e = 0.f;
    const float beta = R.b - R.a * g2;
    const float mu = R.c - R.a * d2 - beta * g1;
    const float inv = rcp(mu);
    chk = fmaf(mu, inv, chk);
    const float g = (R.d - beta * d1) * inv, dl = R.e * inv;
    const float zf = (f - R.a * zf2 - beta * zf1) * inv;
    const float za = ((i == 0 ? 1.f : 0.f) - R.a * za2 - beta * za1) * inv;
    const float zb = ((i == 1 ? 1.f : 0.f) - R.a * zb2 - beta * zb1) * inv;
    if (i == m - 2) {
      gm2 = g;
      im2 = inv;
    }
    bm1 = beta;
    im1 = inv;
    g2 = g1;
    d2 = d1;
    g1 = g;
    d1 = dl;
    zf2 = zf1;
    zf1 = zf;
    za2 = za1;
    za1 = za;
    zb2 = zb1;
    zb1 = zb;
  }
  // back substitution of the last two rows: x_{m-1} = z_{m-1},
  // x_{m-2} = z_{m-2} - g_{m-2} x_{m-1}
  X[1][0] = zf1;
  X[1][1] = za1;
  X[1][2] = zb1;
  X[0][0] = zf2 - gm2 * zf1;
  X[0][1] = za2 - gm2 * za1;
  X[0][2] = zb2 - gm2 * zb1;
  // e_{m-2}: z_{m-2} = 1/mu_{m-2}, z_{m-1} = -beta_{m-1} z_{m-2}/mu_{m-1};
  // e_{m-1}: z_{m-1} = 1/mu_{m-1}
  X[1][3] = -bm1 * im2 * im1;
  X[0][3] = im2 - gm2 * X[1][3];
  X[1][4] = im1;
  X[0][4] = -gm2 * im1;
  if (!(chk == chk)) bad = 1;
}

// The record of one line of segment k (see the file comment): for the
// separator k (own: values 0..9, written by segment k) and separator k + 1
// (next: values 10..19 of separator k + 1, written by segment k).
//   own:  Dp = A_ss - T M_FF P (4), U = -T M_FL Q (4), rp = f_s - T y_F (2)
//   next: Lw = -R M_LF P (4), Dm = -R M_LL Q (4), rm = -R y_L (2)
// with P, Q the interior's couplings to its left and right separators, T
// and R the separators' couplings into the interior, A_ss the separator's
// own 2 x 2 block.  XF, XL: the two passes' results (XF of the reversed
// pass).  Cells are local (0 = the segment's first cell); p1 = segment
// length; the band holds cells 0 .. p1 + 1.
template <int NL, class RhsF>
__device__ __forceinline__ void write_record(const float* band, int line, int k, int S, int p1, const float XL[2][5],
                                             const float XF[2][5], RhsF RHS, float* rec, size_t nlines,
                                             size_t gline) {
  auto B = [&](int cell, int q) { return band[(cell * 5 + q) * NL + line]; };
  const int p0 = k > 0 ? 2 : 0;
  // original rows 0, 1 of the interior = reversed rows m-1, m-2
  const float yF0 = XF[1][0], yF1 = XF[0][0];
  const M2 MFF = mk2(XF[1][4], XF[1][3], XF[0][4], XF[0][3]);
  const M2 MFL = mk2(XF[1][2], XF[1][1], XF[0][2], XF[0][1]);
  const float yL0 = XL[0][0], yL1 = XL[1][0];
  const M2 MLF = mk2(XL[0][1], XL[0][2], XL[1][1], XL[1][2]);
  const M2 MLL = mk2(XL[0][3], XL[0][4], XL[1][3], XL[1][4]);
  const M2 P = mk2(B(p0, 0), B(p0, 1), 0.f, B(p0 + 1, 0));
  const bool next = k + 1 < S;
  const M2 Q = next ? mk2(B(p1 - 2, 4), 0.f, B(p1 - 1, 3), B(p1 - 1, 4)) : mk2(0.f, 0.f, 0.f, 0.f);
  if (k > 0) {
    const M2 T = mk2(B(0, 4), 0.f, B(1, 3), B(1, 4));
    const M2 Ass = mk2(B(0, 2), B(0, 3), B(1, 1), B(1, 2));
    const M2 Dp = sub2(Ass, mul2(mul2(T, MFF), P));
    const M2 U = mul2(mul2(T, MFL), Q);  // negated below
    float t0, t1;
    mv2(T, yF0, yF1, t0, t1);
    float* o = rec + ((size_t)(k - 1) * kRec) * nlines + gline;
    const float v[10] = {Dp.a, Dp.b, Dp.c, Dp.d, -U.a, -U.b, -U.c, -U.d, RHS(0) - t0, RHS(1) - t1};
#pragma unroll
    for (int q = 0; q < 10; ++q) o[q * nlines] = v[q];
  }
  if (next) {
    const M2 R = mk2(B(p1, 0), B(p1, 1), 0.f, B(p1 + 1, 0));
    const M2 Lw = k > 0 ? mul2(mul2(R, MLF), P) : mk2(0.f, 0.f, 0.f, 0.f);
    const M2 Dm = mul2(mul2(R, MLL), Q);
    float t0, t1;
    mv2(R, yL0, yL1, t0, t1);
    float* o = rec + ((size_t)k * kRec + 10) * nlines + gline;
    const float v[10] = {-Lw.a, -Lw.b, -Lw.c, -Lw.d, -Dm.a, -Dm.b, -Dm.c, -Dm.d, -t0, -t1};
#pragma unroll
    for (int q = 0; q < 10; ++q) o[q * nlines] = v[q];
  }
}

// Phase 3 for the lines of a tile: the interior [p0, p1) of every line
// solved with the separators' values on the right side, by a twisted LU:
// thread role 0 eliminates rows 0..h-1 top-down, role 1 rows m-1..h
// bottom-up, a 4 x 4 seam solve gives x_{h-2..h+1}, and both substitute
// back outward (m >= 4; shorter interiors: role 0 alone).  Factors (g, dl,
// z) overwrite the band slots a, b, c of each row.  All threads of the
// block must call it (it synchronises).  Lines line0 + lane of role r are
// handled by threads [r * NL, (r + 1) * NL).  RHS(line, i): right side of
// interior row i (separator terms included).  PUT(line, i, x): solution.
template <int NL>
struct Seam {
  LUState<float> top[NL], bot[NL];
  float x[NL][4];
};
template <int NL, class RhsF, class PutF>
__device__ __forceinline__ void twisted_solve(float* band, Seam<NL>& SM, int nl, int p0, int m, RhsF RHS, PutF PUT,
                                              int& bad) {
  const int t = threadIdx.x, role = t / NL, line = t % NL;
  const bool act = role < 2 && line < nl;
  const bool tw = m >= 4;
  const int h = tw ? m / 2 : m;
  LUState<float> lu;
  lu.reset();
  float chk = 0.f;
  auto fac = [&](int i) { return band + (p0 + i) * 5 * NL + line; };
  auto row_nat = [&](int i) {
    Row R = band_row<NL>(band, p0 + i, line, false);
    if (i == 0) R.b = 0.f;
    if (i <= 1) R.a = 0.f;
    if (i + 1 >= m) R.d = 0.f;
    if (i + 2 >= m) R.e = 0.f;
    return R;
  };
  if (act && role == 0) {
#pragma unroll 4
    for (int i = 0; i < h; ++i) {
      const Row R = row_nat(i);
      float g, dl, z;
      lu.step(R.a, R.b, R.c, R.d, R.e, RHS(line, i), g, dl, z, chk);
      float* q = fac(i);
      q[0] = g;
      q[NL] = dl;
      q[2 * NL] = z;
    }
    SM.top[line] = lu;
  }
  if (act && role == 1 && tw) {
#pragma unroll 4
    for (int i = m - 1; i >= h; --i) {
      const Row R = row_nat(i);
      float g, dl, z;
      lu.step(R.e, R.d, R.c, R.b, R.a, RHS(line, i), g, dl, z, chk);
      float* q = fac(i);
      q[0] = g;
      q[NL] = dl;
      q[2 * NL] = z;
    }
    SM.bot[line] = lu;
  }
  __syncthreads();
  if (act && role == 0 && tw) {
    float x[4] = {0.f, 0.f, 0.f, 0.f};
    if (!seam(SM.top[line], SM.bot[line], x)) bad = 1;
    for (int q = 0; q < 4; ++q) SM.x[line][q] = x[q];
  }
  __syncthreads();
  if (act && role == 0) {
    float x1, x2;
    int i0;
    if (tw) {
      x2 = SM.x[line][1];  // x_{h-1}
      x1 = SM.x[line][0];  // x_{h-2}
      PUT(line, h - 1, x2);
      PUT(line, h - 2, x1);
      i0 = h - 3;
      float xa = x1, xb = x2;  // x_{i+1}, x_{i+2}
#pragma unroll 4
      for (int i = i0; i >= 0; --i) {
        const float* q = fac(i);
        const float x = q[2 * NL] - q[0] * xa - q[NL] * xb;
        PUT(line, i, x);
        xb = xa;
        xa = x;
      }
    } else {
      float xa = 0.f, xb = 0.f;
#pragma unroll 4
      for (int i = h - 1; i >= 0; --i) {
        const float* q = fac(i);
        const float x = q[2 * NL] - q[0] * xa - q[NL] * xb;
        PUT(line, i, x);
        xb = xa;
        xa = x;
      }
    }
    if (!(chk == chk)) bad = 1;
  }
  if (act && role == 1 && tw) {
    float xa = SM.x[line][3], xb = SM.x[line][2];  // x_{h+1}, x_h
    PUT(line, h, xb);
    PUT(line, h + 1, xa);
#pragma unroll 4
    for (int i = h + 2; i < m; ++i) {
      const float* q = fac(i);
      const float x = q[2 * NL] - q[0] * xa - q[NL] * xb;
      PUT(line, i, x);
      xb = xa;
      xa = x;
    }
    if (!(chk == chk)) bad = 1;
  }
}

// Iteration accumulators shared by all blocks (max and or are
// order-independent, so atomics keep the results deterministic).
struct Acc {
  unsigned err_bits;  // max |v / u_k| as the bits of a non-negative float (NaN is largest)
  int nonfinite;
  int pivot;
  int pad;
};

__device__ __forceinline__ void flag_bad(Acc* acc, int bad) {
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&acc->pivot, 1);
}

// ---------------------------------------------------------------------------
// Film tiles.  The FP32 film of the power-law path is the truncated leading
// float of each height (what the residual kernel writes).  Tiles hold
// wall-reflected values (eq. BoundaryConditions), so a missing neighbour
// equals the cell itself.

template <int P>
__device__ __forceinline__ void load_film_f32(float* dst, const float* __restrict__ src, int row0, int nr, int col0,
                                              int nc, int ny, int nx) {
  for (int k = threadIdx.x; k < nr * nc; k += kT) {
    const int r = k / nc, c = k - r * nc;
    dst[r * P + c] = __ldg(src + (size_t)reflect_index(row0 + r, ny) * nx + reflect_index(col0 + c, nx));
  }
}
template <int P>
__device__ __forceinline__ void load_film_f64(float* dst, const double* __restrict__ src, int row0, int nr, int col0,
                                              int nc, int ny, int nx) {
  for (int k = threadIdx.x; k < nr * nc; k += kT) {
    const int r = k / nc, c = k - r * nc;
    dst[r * P + c] =
        f32_of_pos_f64_fast(__ldg(src + (size_t)reflect_index(row0 + r, ny) * nx + reflect_index(col0 + c, nx)));
  }
}
// rows [row0, row0 + nr) x columns [col0, col0 + nc) inside the grid
template <int P>
__device__ __forceinline__ void load_block(float* dst, const float* __restrict__ src, int row0, int nr, int col0,
                                           int nc, int nx) {
  for (int k = threadIdx.x; k < nr * nc; k += kT) {
    const int r = k / nc, c = k - r * nc;
    dst[r * P + c] = __ldg(src + (size_t)(row0 + r) * nx + col0 + c);
  }
}

// ---------------------------------------------------------------------------
// x phase 1: tile of kRX rows x x segment blockIdx.x (the block exists only
// for grids with more than one x segment).

struct X1Smem {
  float film[(kRX + 2) * (kLX + 7)];   // rows j0-1.., cols c0-2.. (pitch kLX + 7, odd)
  float rt[kRX * (kLX + 1)];           // right side [row][cell]
  float band[(kLX + 2) * 5 * kRX];     // cells c0 .. c1+1
  float X[2][kRX][10];
};

__global__ void __launch_bounds__(kT, 3)
    k_part_x1(ModelK M, LineK<float> L, const float* __restrict__ ul, const float* __restrict__ r,
              float* __restrict__ rec, Acc* __restrict__ acc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  X1Smem& S = *reinterpret_cast<X1Smem*>(smem_raw);
  constexpr int FP = kLX + 7, RP = kLX + 1;
  const int nx = M.nx, ny = M.ny, nS = seg_count<kLX>(nx);
  const int k = blockIdx.x, j0 = blockIdx.y * kRX;
  const int c0 = seg_start<kLX>(k, nx), c1 = seg_end<kLX>(k, nx), len = c1 - c0;
  const bool next = k + 1 < nS;
  const int ncell = len + (next ? 2 : 0);
  const int nrow = min(kRX, ny - j0);
  load_film_f32<FP>(S.film, ul, j0 - 1, nrow + 2, c0 - 2, ncell + 4, ny, nx);
  load_block<RP>(S.rt, r, j0, nrow, c0, len, nx);
  __syncthreads();
  auto film = [&](int line, int cell, int dr, int dc) {
    return S.film[(line + 1 + dr) * FP + (cell - c0 + 2 + dc)];
  };
  build_band<kRX>(L, S.band, nrow, c0, ncell, nx, film);
  __syncthreads();
  const int p0 = k > 0 ? 2 : 0, m = len - p0;
  const int t = threadIdx.x, line = t & 31, dir = t >> 5;
  int bad = 0;
  if (dir < 2 && line < nrow) {
    float X[2][5];
    if (dir == 0) {
      elim_pass([&](int i) { return band_row<kRX>(S.band, p0 + i, line, false); },
                [&](int i) { return S.rt[line * RP + p0 + i]; }, m, X, bad);
    } else {
      elim_pass([&](int i) { return band_row<kRX>(S.band, p0 + m - 1 - i, line, true); },
                [&](int i) { return S.rt[line * RP + p0 + m - 1 - i]; }, m, X, bad);
    }
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 5; ++b) S.X[dir][line][a * 5 + b] = X[a][b];
  }
  if (dir < 2) flag_bad(acc, bad);
  __syncthreads();
  if (dir == 0 && line < nrow) {
    float XL[2][5], XF[2][5];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 5; ++b) {
        XL[a][b] = S.X[0][line][a * 5 + b];
        XF[a][b] = S.X[1][line][a * 5 + b];
      }
    write_record<kRX>(S.band, line, k, nS, len, XL, XF, [&](int i) { return S.rt[line * RP + i]; }, rec,
                      (size_t)ny, (size_t)(j0 + line));
  }
}

// ---------------------------------------------------------------------------
// Phase 2: the reduced block-tridiagonal system of every line (one thread
// per line).  rec is [S-1][kRec][nlines]; the forward sweep overwrites
// values 10..15 of each separator with W^-1 and the reduced right side.
// xs receives the separators' values, [S-1][2][nlines].

__global__ void __launch_bounds__(128)
    k_part_red(float* __restrict__ rec, int nS, int nlines, float* __restrict__ xs, Acc* __restrict__ acc) {
  const int line = blockIdx.x * blockDim.x + threadIdx.x;
  int bad = 0;
  if (line < nlines) {
    const size_t NL = (size_t)nlines;
    M2 Wi = mk2(0.f, 0.f, 0.f, 0.f), Up = mk2(0.f, 0.f, 0.f, 0.f);
    float g0 = 0.f, g1 = 0.f;
    for (int s = 1; s < nS; ++s) {
      float* R = rec + (size_t)(s - 1) * kRec * NL + line;
      float v[kRec];
#pragma unroll
      for (int q = 0; q < kRec; ++q) v[q] = R[q * NL];
      M2 D = mk2(v[0] + v[14], v[1] + v[15], v[2] + v[16], v[3] + v[17]);
      float h0 = v[8] + v[18], h1 = v[9] + v[19];
      if (s >= 2) {
        const M2 Lam = mul2(mk2(v[10], v[11], v[12], v[13]), Wi);
        D = sub2(D, mul2(Lam, Up));
        float l0, l1;
        mv2(Lam, g0, g1, l0, l1);
        h0 -= l0;
        h1 -= l1;
      }
      const float det = D.a * D.d - D.b * D.c;
      const float id = 1.f / det;
      if (!(det != 0.f) || !(id - id == 0.f)) bad = 1;
      Wi = mk2(D.d * id, -D.b * id, -D.c * id, D.a * id);
      Up = mk2(v[4], v[5], v[6], v[7]);
      g0 = h0;
      g1 = h1;
      R[10 * NL] = Wi.a;
      R[11 * NL] = Wi.b;
      R[12 * NL] = Wi.c;
      R[13 * NL] = Wi.d;
      R[14 * NL] = g0;
      R[15 * NL] = g1;
    }
    // back substitution: x_s = W_s^-1 (g_s - U_s x_{s+1})
    float x0 = 0.f, x1 = 0.f;
    for (int s = nS - 1; s >= 1; --s) {
      const float* R = rec + (size_t)(s - 1) * kRec * NL + line;
      float h0 = R[14 * NL], h1 = R[15 * NL];
      if (s + 1 < nS) {
        float u0, u1;
        mv2(mk2(R[4 * NL], R[5 * NL], R[6 * NL], R[7 * NL]), x0, x1, u0, u1);
        h0 -= u0;
        h1 -= u1;
      }
      mv2(mk2(R[10 * NL], R[11 * NL], R[12 * NL], R[13 * NL]), h0, h1, x0, x1);
      float* o = xs + (size_t)(s - 1) * 2 * NL + line;
      o[0] = x0;
      o[NL] = x1;
    }
  }
  flag_bad(acc, bad);
}

// ---------------------------------------------------------------------------
// x phase 3 + y phase 1: tile = y segment blockIdx.y x x segment blockIdx.x.

struct XYSmem {
  float film[(kLY + 6) * (kLX + 5)];   // rows r0-2 .. r1+3, cols c0-2 .. c1+1 (pitch kLX + 5)
  float wt[kLY * (kLX + 1)];           // right side r, then w, [row][col]
  // x band [cell < kLX][5][row < kLY], then y band [cell < kLY + 2][5][col < kLX]
  float band[(kLX * kLY > (kLY + 2) * kLX ? kLX * kLY : (kLY + 2) * kLX) * 5];
  Seam<kLY> seam;
  float xsl[kLY][2], xsr[kLY][2];
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
  load_film_f32<FP>(S.film, ul, r0 - 2, nrowy + 4, c0 - 2, nc + 4, ny, nx);
  load_block<WP>(S.wt, rw, r0, nr, c0, nc, nx);
  for (int q = threadIdx.x; q < 2 * nr; q += kT) {
    const int row = q >> 1, e = q & 1;
    S.xsl[row][e] = kx > 0 ? xsx[((size_t)(kx - 1) * 2 + e) * ny + r0 + row] : 0.f;
    S.xsr[row][e] = kx + 1 < nSx ? xsx[((size_t)kx * 2 + e) * ny + r0 + row] : 0.f;
  }
  __syncthreads();
  // ---- x band of the tile's rows, cells c0 .. c1-1
  {
    auto film = [&](int line, int cell, int dr, int dc) {
      return S.film[(line + 2 + dr) * FP + (cell - c0 + 2 + dc)];
    };
    build_band<kLY>(L, S.band, nr, c0, nc, nx, film);
  }
  __syncthreads();
  int bad = 0;
  // ---- x phase 3: interiors of the tile's rows; separators from phase 2
  {
    const int p0 = kx > 0 ? 2 : 0, m = nc - p0;
    const bool right = kx + 1 < nSx;
    auto B = [&](int cell, int q, int line) { return S.band[(cell * 5 + q) * kLY + line]; };
    auto rhs = [&](int line, int i) {
      const int cell = p0 + i;
      float f = S.wt[line * WP + cell];
      if (kx > 0) {
        if (i == 0) f -= B(cell, 0, line) * S.xsl[line][0] + B(cell, 1, line) * S.xsl[line][1];
        if (i == 1) f -= B(cell, 0, line) * S.xsl[line][1];
      }
      if (right) {
        if (i == m - 2) f -= B(cell, 4, line) * S.xsr[line][0];
        if (i == m - 1) f -= B(cell, 3, line) * S.xsr[line][0] + B(cell, 4, line) * S.xsr[line][1];
      }
      return f;
    };
    auto put = [&](int line, int i, float x) { S.wt[line * WP + p0 + i] = x; };
    twisted_solve<kLY>(S.band, S.seam, nr, p0, m, rhs, put, bad);
    if (kx > 0)
      for (int q = threadIdx.x; q < 2 * nr; q += kT) S.wt[(q >> 1) * WP + (q & 1)] = S.xsl[q >> 1][q & 1];
  }
  __syncthreads();
  // ---- store w; y band of the tile's columns, rows r0 .. r1 (+ next separator)
  for (int k = threadIdx.x; k < nr * nc; k += kT) {
    const int rr = k / nc, cc = k - rr * nc;
    rw[(size_t)(r0 + rr) * nx + c0 + cc] = S.wt[rr * WP + cc];
  }
  {
    auto film = [&](int line, int cell, int dr, int dc) {
      return S.film[(cell - r0 + 2 + dr) * FP + (line + 2 + dc)];
    };
    build_band<kLX>(L, S.band, nc, r0, nrowy, ny, film);
  }
  __syncthreads();
  // ---- y phase 1 (lines = the tile's columns)
  if (nSy > 1) {
    float(*X)[kLX][10] = reinterpret_cast<float(*)[kLX][10]>(S.film);  // film no longer needed
    const int t = threadIdx.x, line = t % kLX, dir = t / kLX;
    const int p0 = ky > 0 ? 2 : 0, m = nr - p0;
    if (dir < 2 && line < nc) {
      float Xv[2][5];
      if (dir == 0)
        elim_pass([&](int i) { return band_row<kLX>(S.band, p0 + i, line, false); },
                  [&](int i) { return S.wt[(p0 + i) * WP + line]; }, m, Xv, bad);
      else
        elim_pass([&](int i) { return band_row<kLX>(S.band, p0 + m - 1 - i, line, true); },
                  [&](int i) { return S.wt[(p0 + m - 1 - i) * WP + line]; }, m, Xv, bad);
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 5; ++b) X[dir][line][a * 5 + b] = Xv[a][b];
    }
    __syncthreads();
    if (dir == 0 && line < nc) {
      float XL[2][5], XF[2][5];
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 5; ++b) {
          XL[a][b] = X[0][line][a * 5 + b];
          XF[a][b] = X[1][line][a * 5 + b];
        }
      write_record<kLX>(S.band, line, ky, nSy, nr, XL, XF, [&](int i) { return S.wt[i * WP + line]; }, recy,
                        (size_t)nx, (size_t)(c0 + line));
    }
  }
  flag_bad(acc, bad);
}

// ---------------------------------------------------------------------------
// y phase 3, Newton update and reductions: tile = y segment blockIdx.y x
// kCY columns from blockIdx.x * kCY.

struct YCSmem {
  float film[(kLY + 4) * (kCY + 3)];   // rows r0-2 .. r1+1, cols i0-1 .. (pitch kCY + 3)
  float wt[kLY * (kCY + 1)];           // w, then v
  float band[kLY * 5 * kCY];
  Seam<kCY> seam;
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
  constexpr int FP = kCY + 3, WP = kCY + 1;
  const int nx = M.nx, ny = M.ny, nSy = seg_count<kLY>(ny);
  const int i0 = blockIdx.x * kCY, ky = blockIdx.y;
  const int nc = min(kCY, nx - i0);
  const int r0 = seg_start<kLY>(ky, ny), r1 = seg_end<kLY>(ky, ny), nr = r1 - r0;
  load_film_f64<FP>(S.film, u, r0 - 2, nr + 4, i0 - 1, nc + 2, ny, nx);
  load_block<WP>(S.wt, w, r0, nr, i0, nc, nx);
  for (int q = threadIdx.x; q < 2 * nc; q += kT) {
    const int col = q >> 1, e = q & 1;
    S.ysl[col][e] = ky > 0 ? xsy[((size_t)(ky - 1) * 2 + e) * nx + i0 + col] : 0.f;
    S.ysr[col][e] = ky + 1 < nSy ? xsy[((size_t)ky * 2 + e) * nx + i0 + col] : 0.f;
  }
  __syncthreads();
  {
    auto film = [&](int line, int cell, int dr, int dc) {
      return S.film[(cell - r0 + 2 + dr) * FP + (line + 1 + dc)];
    };
    build_band<kCY>(L, S.band, nc, r0, nr, ny, film);
  }
  __syncthreads();
  int bad = 0;
  {
    const int p0 = ky > 0 ? 2 : 0, m = nr - p0;
    const bool right = ky + 1 < nSy;
    auto B = [&](int cell, int q, int line) { return S.band[(cell * 5 + q) * kCY + line]; };
    auto rhs = [&](int line, int i) {
      const int cell = p0 + i;
      float f = S.wt[cell * WP + line];
      if (ky > 0) {
        if (i == 0) f -= B(cell, 0, line) * S.ysl[line][0] + B(cell, 1, line) * S.ysl[line][1];
        if (i == 1) f -= B(cell, 0, line) * S.ysl[line][1];
      }
      if (right) {
        if (i == m - 2) f -= B(cell, 4, line) * S.ysr[line][0];
        if (i == m - 1) f -= B(cell, 3, line) * S.ysr[line][0] + B(cell, 4, line) * S.ysr[line][1];
      }
      return f;
    };
    auto put = [&](int line, int i, float x) { S.wt[(p0 + i) * WP + line] = x; };
    twisted_solve<kCY>(S.band, S.seam, nc, p0, m, rhs, put, bad);
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

}  // namespace part
}  // namespace tf
