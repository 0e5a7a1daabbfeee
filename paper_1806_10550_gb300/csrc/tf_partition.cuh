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
// Every per-line operation here runs on two lines at once, one in each lane
// of the paired FP32 instructions (float2 add/mul/fma): band rows, the
// elimination passes and the interior solves.  Only the 4 x 4 seam solves,
// which pivot, run one line at a time.
//
// This header holds the device building blocks (the (3, 2) power law); the
// kernels are in tf_part.cu:
//   x phase 1 on a tile of 32 rows x one x segment, from the FP32 film and
//              the right side r = -G written by the residual kernel;
//   phase 2 of one direction, one warp per line;
//   x phase 3 on a tile of one y segment x one x segment (writes w), then
//              y phase 1 on the same tile's columns;
//   y phase 3 on a tile of one y segment x 64 columns, the Newton update
//              u_{k+1} = u_k + v and the iteration's reductions.
#pragma once

#include "tf_line_sweeps.cuh"

namespace tf {

// paired FP32 operations (one IEEE operation per lane)
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_neg(float2 a) { return make_float2(-a.x, -a.y); }
// a - b as fma(b, -1, a): the same IEEE result as a + (-b) (the product
// b * -1 is exact), in one paired instruction with no separate negation of
// b.  (A PTX sub.rn.f32x2 was contracted with a preceding paired multiply,
// which breaks the error-free transformations built on it.)
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 p_splat(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 p_rcp(float2 a) { return make_float2(rcp(a.x), rcp(a.y)); }

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

// 2 x 2 matrices, row-major [[a, b], [c, d]] (one line; phase 2 and records)
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

// ---------------------------------------------------------------------------
// Band rows of two lines.  Layout in shared memory: band[(cell * 5 + q) *
// NL + line], q = a..e (multiplying x_{i-2}..x_{i+2}); lines 2p and 2p + 1
// are one float2.

struct Row2 {
  float2 a, b, c, d, e;
};
template <int NL>
__device__ __forceinline__ Row2 band_row2(const float* band, int cell, int pair, bool rev) {
  const float2* p = reinterpret_cast<const float2*>(band + cell * 5 * NL) + pair;
  constexpr int Q = NL / 2;
  Row2 r;
  if (!rev) {
    r.a = p[0];
    r.b = p[Q];
    r.c = p[2 * Q];
    r.d = p[3 * Q];
    r.e = p[4 * Q];
  } else {
    r.e = p[0];
    r.d = p[Q];
    r.c = p[2 * Q];
    r.b = p[3 * Q];
    r.a = p[4 * Q];
  }
  return r;
}

// Per-cell film values of the (n, m) = (3, 2) power law, pre-scaled for the
// band (the constants of LineK, as cell_pl32): F0 = k3 C h^3, F1 = k1 A1 -
// k1 B1 / h, D0 = (k1/ds^2) 3 C h^2, D1 = k1 B1 / h^2, and the unscaled
// Laplacian.
struct LineK2 {
  float2 pF0, pF1a, pF1b, pD0, pD1;
};
__device__ __forceinline__ LineK2 pack_consts(const LineK<float>& L) {
  LineK2 K;
  K.pF0 = p_splat(L.pF0);
  K.pF1a = p_splat(L.pF1a);
  K.pF1b = p_splat(L.pF1b);
  K.pD0 = p_splat(L.pD0);
  K.pD1 = p_splat(L.pD1);
  return K;
}
struct Cell2 {
  float2 u, lap, F0, F1, D0, D1;
};
template <class Acc>
__device__ __forceinline__ Cell2 cell2(const LineK2& K, Acc U) {
  Cell2 X;
  const float2 uc = U(0, 0);
  X.u = uc;
  X.lap = p_add(p_add(p_sub(U(0, 1), uc), p_sub(U(0, -1), uc)), p_add(p_sub(U(1, 0), uc), p_sub(U(-1, 0), uc)));
  const float2 s = p_rcp(uc), h2 = p_mul(uc, uc);
  X.F0 = p_mul(K.pF0, p_mul(h2, uc));
  X.F1 = p_fma(p_neg(K.pF1b), s, K.pF1a);
  X.D0 = p_mul(K.pD0, h2);
  X.D1 = p_mul(K.pD1, p_mul(s, s));
  return X;
}
// derivatives of the scaled flux through the face between line cells p and
// q = p + 1 (see face_scaled): pl, qr say whether p has a left and q a right
// neighbour (walls fold the reflected cells away)
__device__ __forceinline__ void face2(const Cell2& P, const Cell2& Q, bool pl, bool qr, float2 dF[4]) {
  const float2 dl = p_sub(Q.lap, P.lap), du = p_sub(Q.u, P.u);
  const float2 c3 = p_add(P.F0, Q.F0), Bd = p_add(P.F1, Q.F1);
  const float2 tp = p_fma(P.D0, dl, p_mul(P.D1, du)), tq = p_fma(Q.D0, dl, p_mul(Q.D1, du));
  const float wp = pl ? 1.f : 0.f, wq = qr ? 1.f : 0.f;
  dF[0] = p_mul(p_splat(-wp), c3);
  dF[1] = p_fma(p_splat(2.f + wp), c3, p_sub(tp, Bd));
  dF[2] = p_fma(p_splat(-(2.f + wq)), c3, p_add(tq, Bd));
  dF[3] = p_mul(p_splat(wq), c3);
}
// Band rows of line cells ia .. ib-1 (at most G) of two lines, from the
// film around them: A(s, dr, dc) gives the film pair at line cell ia + s
// offset by (dr, dc).  Faces outside 0..n-1 carry nothing.  OUT(s, row).
// Rolling: two cells and two faces live at a time.
template <int G, class Acc, class Out>
__device__ __forceinline__ void band_rows2(const LineK2& K, Acc A, int ia, int ib, int n, Out out) {
  auto face_at = [&](const Cell2& P, const Cell2& Q, int f, float2 F[4]) {  // cells ia+f-1 | ia+f
    const int q = ia + f - 1;
    face2(P, Q, q > 0, q + 2 < n, F);
    if (!(q >= 0 && q + 1 < n))
      for (int k = 0; k < 4; ++k) F[k] = p_splat(0.f);
  };
  Cell2 Cp = cell2(K, [&](int dr, int dc) { return A(-1, dr, dc); });
  Cell2 Cq = cell2(K, [&](int dr, int dc) { return A(0, dr, dc); });
  float2 Fa[4], Fb[4];
  face_at(Cp, Cq, 0, Fa);
#pragma unroll
  for (int s = 0; s < G; ++s) {
    Cp = Cq;
    Cq = cell2(K, [&](int dr, int dc) { return A(s + 1, dr, dc); });
    face_at(Cp, Cq, s + 1, Fb);
    if (ia + s < ib) {
      Row2 R;
      R.a = p_neg(Fa[0]);
      R.b = p_sub(Fb[0], Fa[1]);
      R.c = p_add(p_splat(1.f), p_sub(Fb[1], Fa[2]));
      R.d = p_sub(Fb[2], Fa[3]);
      R.e = Fb[3];
      out(s, R);
    }
    for (int k = 0; k < 4; ++k) Fa[k] = Fb[k];
  }
}

// Build the band rows of cells [ia0, ia0 + ncell) of the nl lines of a tile
// (NL lines at most, in pairs) with NT threads.  film(pair, cell, dr, dc)
// gives the film of lines 2 pair, 2 pair + 1 at line cell `cell` (global
// index along the line), offset by dr across and dc along the line.
template <int NL, int NT, class Film>
__device__ __forceinline__ void build_band(const LineK2& K, float* band, int nl, int ia0, int ncell, int n,
                                           Film film) {
  constexpr int NP = NL / 2;
  const int ngrp = (ncell + kGB - 1) / kGB, npair = (nl + 1) / 2;
  for (int task = threadIdx.x; task < ngrp * NP; task += NT) {
    const int pair = task % NP, grp = task / NP;
    if (pair >= npair) continue;
    const int ia = ia0 + grp * kGB, ib = min(ia0 + ncell, ia + kGB);
    auto A = [&](int s, int dr, int dc) { return film(pair, ia + s, dr, dc); };
    float2* P = reinterpret_cast<float2*>(band + (ia - ia0) * 5 * NL) + pair;
    auto out = [&](int s, const Row2& R) {
      float2* q = P + s * 5 * NP;
      q[0] = R.a;
      q[NP] = R.b;
      q[2 * NP] = R.c;
      q[3 * NP] = R.d;
      q[4 * NP] = R.e;
    };
    band_rows2<kGB>(K, A, ia, ib, n, out);
  }
}

// ---------------------------------------------------------------------------
// Phase 1: one elimination pass over an interior of m >= 2 rows of two
// lines, LU without pivoting of the interior's own matrix (entries that
// reach outside it dropped), with the right sides f and the unit vectors
// e_0, e_1.  X receives rows m-2 and m-1 (in the pass's orientation) of
// A^-1 applied to [f, e_0, e_1, e_{m-2}, e_{m-1}].  ROW(i) gives row i in
// the pass's orientation; RHS(i) its right side.  A zero or non-finite
// pivot sets bad.
template <class RowF, class RhsF>
__device__ __forceinline__ void elim_pass2(RowF ROW, RhsF RHS, int m, float2 X[2][5], int& bad, bool two) {
  const float2 z0 = p_splat(0.f), one = p_splat(1.f);
  float2 g1 = z0, d1 = z0, g2 = z0, d2 = z0;
  float2 zf1 = z0, zf2 = z0, za1 = z0, za2 = z0, zb1 = z0, zb2 = z0;
  float2 gm2 = z0, im2 = z0, bm1 = z0, im1 = z0, chk = z0;
  for (int i = 0; i < m; ++i) {
    Row2 R = ROW(i);
    const float2 f = RHS(i);
    // rows 0 and 1 lose the entries reaching left of the interior, rows
    // m-2 and m-1 those reaching right of it
    if (i == 0) R.b = z0;
    if (i <= 1) R.a = z0;
    if (i + 1 >= m) R.d = z0;
    if (i + 2 >= m) R.e = z0;
    const float2 beta = p_fma(p_neg(R.a), g2, R.b);
    const float2 mu = p_fma(p_neg(beta), g1, p_fma(p_neg(R.a), d2, R.c));
    const float2 inv = p_rcp(mu);
    chk = p_fma(mu, inv, chk);
    const float2 g = p_mul(p_fma(p_neg(beta), d1, R.d), inv), dl = p_mul(R.e, inv);
    const float2 zf = p_mul(p_fma(p_neg(beta), zf1, p_fma(p_neg(R.a), zf2, f)), inv);
    const float2 za = p_mul(p_fma(p_neg(beta), za1, p_fma(p_neg(R.a), za2, i == 0 ? one : z0)), inv);
    const float2 zb = p_mul(p_fma(p_neg(beta), zb1, p_fma(p_neg(R.a), zb2, i == 1 ? one : z0)), inv);
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
  X[0][0] = p_fma(p_neg(gm2), zf1, zf2);
  X[0][1] = p_fma(p_neg(gm2), za1, za2);
  X[0][2] = p_fma(p_neg(gm2), zb1, zb2);
  // e_{m-2}: z_{m-2} = 1/mu_{m-2}, z_{m-1} = -beta_{m-1} z_{m-2}/mu_{m-1};
  // e_{m-1}: z_{m-1} = 1/mu_{m-1}
  X[1][3] = p_mul(p_neg(bm1), p_mul(im2, im1));
  X[0][3] = p_fma(p_neg(gm2), X[1][3], im2);
  X[1][4] = im1;
  X[0][4] = p_mul(p_neg(gm2), im1);
  if (!(chk.x == chk.x) || (two && !(chk.y == chk.y))) bad = 1;  // two: the second line exists
}

// The record of one line of segment k (see the file comment): for the
// separator k (own: values 0..9, written by segment k) and separator k + 1
// (next: values 10..19 of separator k + 1, written by segment k).  Records
// are stored rec[separator - 1][20][line]: a warp over 32 consecutive lines
// reads each value of a row with one coalesced access.
//   own:  Dp = A_ss - T M_FF P (4), U = -T M_FL Q (4), rp = f_s - T y_F (2)
//   next: Lw = -R M_LF P (4), Dm = -R M_LL Q (4), rm = -R y_L (2)
// with P, Q the interior's couplings to its left and right separators, T
// and R the separators' couplings into the interior, A_ss the separator's
// own 2 x 2 block.  XF, XL: the two passes' results for this line (XF of
// the reversed pass).  Cells are local (0 = the segment's first cell); p1 =
// segment length; the band holds cells 0 .. p1 + 1.
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
    float* o = rec + (size_t)(k - 1) * kRec * nlines + gline;
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

// Phase 1 of a tile after its band: warp 0 (one thread per pair of lines)
// runs the forward pass, warp 1 the reversed one, over the interior of every
// line of segment k (len cells); then one thread per line writes the
// records.  RHS(line, cell) is the right side of the line's local cell.
// X: scratch [2][NL][10].  All threads of the block call it (it
// synchronises).
template <int NL, class RhsF>
__device__ __forceinline__ void phase1(const float* band, float (*X)[NL][10], int nl, int k, int S, int len,
                                       RhsF RHS, float* rec, size_t nlines, size_t gline0, int& bad) {
  constexpr int NP = NL / 2;
  static_assert(NP <= 32, "one warp per pass direction");
  // the two directions run in different warps (no divergence between them)
  const int t = threadIdx.x, pair = t & 31, dir = t >> 5;
  const int p0 = k > 0 ? 2 : 0, m = len - p0;
  if (dir < 2 && pair < NP && 2 * pair < nl) {
    auto rhs2 = [&](int cell) { return make_float2(RHS(2 * pair, cell), RHS(2 * pair + 1, cell)); };
    float2 Xv[2][5];
    const bool two = 2 * pair + 1 < nl;
    if (dir == 0)
      elim_pass2([&](int i) { return band_row2<NL>(band, p0 + i, pair, false); },
                 [&](int i) { return rhs2(p0 + i); }, m, Xv, bad, two);
    else
      elim_pass2([&](int i) { return band_row2<NL>(band, p0 + m - 1 - i, pair, true); },
                 [&](int i) { return rhs2(p0 + m - 1 - i); }, m, Xv, bad, two);
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 5; ++b) {
        X[dir][2 * pair][a * 5 + b] = Xv[a][b].x;
        X[dir][2 * pair + 1][a * 5 + b] = Xv[a][b].y;
      }
  }
  __syncthreads();
  if (t < nl) {
    float XL[2][5], XF[2][5];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 5; ++b) {
        XL[a][b] = X[0][t][a * 5 + b];
        XF[a][b] = X[1][t][a * 5 + b];
      }
    write_record<NL>(band, t, k, S, len, XL, XF, [&](int i) { return RHS(t, i); }, rec, nlines, gline0 + t);
  }
}

// ---------------------------------------------------------------------------
// Phase 3 for the lines of a tile: the interior [p0, p0+m) of every line
// solved with the separators' values on the right side, by a twisted LU:
// role 0 eliminates rows 0..h-1 top-down, role 1 rows m-1..h bottom-up, a
// 4 x 4 seam solve gives x_{h-2..h+1}, and both substitute back outward
// (m >= 4; shorter interiors: role 0 alone).  Each thread carries two lines
// (a pair).  Factors (g, dl, z) overwrite the band slots a, b, c of each
// row.  All threads of the block must call it (it synchronises).  Role r
// is warp r, one thread per pair of lines.  RHS(pair, i): right side of
// interior row i (separator terms included).  PUT(pair, i, x): solution.

struct LU2 {
  float2 g1, d1, z1, g2, d2, z2;
};
template <int NL>
struct Seam2 {
  LU2 top[NL / 2], bot[NL / 2];
  float x[NL][4];
};
__device__ __forceinline__ void lu2_step(LU2& s, const Row2& R, float2 r, float2& g, float2& dl, float2& z,
                                         float2& chk) {
  const float2 beta = p_fma(p_neg(R.a), s.g2, R.b);
  const float2 mu = p_fma(p_neg(beta), s.g1, p_fma(p_neg(R.a), s.d2, R.c));
  const float2 inv = p_rcp(mu);
  g = p_mul(p_fma(p_neg(beta), s.d1, R.d), inv);
  dl = p_mul(R.e, inv);
  z = p_mul(p_fma(p_neg(beta), s.z1, p_fma(p_neg(R.a), s.z2, r)), inv);
  s.g2 = s.g1;
  s.d2 = s.d1;
  s.z2 = s.z1;
  s.g1 = g;
  s.d1 = dl;
  s.z1 = z;
  chk = p_fma(mu, inv, chk);
}
__device__ __forceinline__ LUState<float> lane_state(const LU2& s, int lane) {
  LUState<float> r;
  r.g1 = lane ? s.g1.y : s.g1.x;
  r.d1 = lane ? s.d1.y : s.d1.x;
  r.z1 = lane ? s.z1.y : s.z1.x;
  r.g2 = lane ? s.g2.y : s.g2.x;
  r.d2 = lane ? s.d2.y : s.d2.x;
  r.z2 = lane ? s.z2.y : s.z2.x;
  return r;
}

template <int NL, class RhsF, class PutF>
__device__ __forceinline__ void twisted_solve2(float* band, Seam2<NL>& SM, int nl, int p0, int m, RhsF RHS, PutF PUT,
                                               int& bad) {
  constexpr int NP = NL / 2;
  static_assert(NP <= 32, "one warp per role");
  // the two roles run in different warps (no divergence between them)
  const int t = threadIdx.x, role = t >> 5, pair = t & 31;
  const bool act = role < 2 && pair < NP && 2 * pair < nl;
  const bool two = 2 * pair + 1 < nl;  // the pair's second line exists
  const bool tw = m >= 4;
  const int h = tw ? m / 2 : m;
  const float2 z0 = p_splat(0.f);
  LU2 lu;
  lu.g1 = lu.d1 = lu.z1 = lu.g2 = lu.d2 = lu.z2 = z0;
  float2 chk = z0;
  auto fac = [&](int i) { return reinterpret_cast<float2*>(band + (p0 + i) * 5 * NL) + pair; };
  auto row_nat = [&](int i) {
    Row2 R = band_row2<NL>(band, p0 + i, pair, false);
    if (i == 0) R.b = z0;
    if (i <= 1) R.a = z0;
    if (i + 1 >= m) R.d = z0;
    if (i + 2 >= m) R.e = z0;
    return R;
  };
  if (act && role == 0) {
    for (int i = 0; i < h; ++i) {
      const Row2 R = row_nat(i);
      float2 g, dl, z;
      lu2_step(lu, R, RHS(pair, i), g, dl, z, chk);
      float2* q = fac(i);
      q[0] = g;
      q[NP] = dl;
      q[2 * NP] = z;
    }
    SM.top[pair] = lu;
  }
  if (act && role == 1 && tw) {
    for (int i = m - 1; i >= h; --i) {
      const Row2 R = row_nat(i);
      Row2 Rr;
      Rr.a = R.e;
      Rr.b = R.d;
      Rr.c = R.c;
      Rr.d = R.b;
      Rr.e = R.a;
      float2 g, dl, z;
      lu2_step(lu, Rr, RHS(pair, i), g, dl, z, chk);
      float2* q = fac(i);
      q[0] = g;
      q[NP] = dl;
      q[2 * NP] = z;
    }
    SM.bot[pair] = lu;
  }
  __syncthreads();
  if (tw && t < nl) {  // one seam per line
    float x[4] = {0.f, 0.f, 0.f, 0.f};
    if (!seam(lane_state(SM.top[t >> 1], t & 1), lane_state(SM.bot[t >> 1], t & 1), x)) bad = 1;
    for (int q = 0; q < 4; ++q) SM.x[t][q] = x[q];
  }
  __syncthreads();
  if (act && role == 0) {
    float2 xa, xb;  // x_{i+1}, x_{i+2}
    int i0;
    if (tw) {
      xa = make_float2(SM.x[2 * pair][0], SM.x[2 * pair + 1][0]);  // x_{h-2}
      xb = make_float2(SM.x[2 * pair][1], SM.x[2 * pair + 1][1]);  // x_{h-1}
      PUT(pair, h - 1, xb);
      PUT(pair, h - 2, xa);
      i0 = h - 3;
    } else {
      xa = xb = z0;
      i0 = h - 1;
    }
    for (int i = i0; i >= 0; --i) {
      const float2* q = fac(i);
      const float2 x = p_fma(p_neg(q[NP]), xb, p_fma(p_neg(q[0]), xa, q[2 * NP]));
      PUT(pair, i, x);
      xb = xa;
      xa = x;
    }
    if (!(chk.x == chk.x) || (two && !(chk.y == chk.y))) bad = 1;
  }
  if (act && role == 1 && tw) {
    float2 xa = make_float2(SM.x[2 * pair][3], SM.x[2 * pair + 1][3]);  // x_{h+1}
    float2 xb = make_float2(SM.x[2 * pair][2], SM.x[2 * pair + 1][2]);  // x_h
    PUT(pair, h, xb);
    PUT(pair, h + 1, xa);
    for (int i = h + 2; i < m; ++i) {
      const float2* q = fac(i);
      const float2 x = p_fma(p_neg(q[NP]), xb, p_fma(p_neg(q[0]), xa, q[2 * NP]));
      PUT(pair, i, x);
      xb = xa;
      xa = x;
    }
    if (!(chk.x == chk.x) || (two && !(chk.y == chk.y))) bad = 1;
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
// equals the cell itself.  R x C tiles (compile-time shape; rows [0, nr)
// and columns [0, nc) filled): inside the grid, pairs of values per thread
// and only constant divisions; at the walls, element by element with
// reflected indices.

template <int R, int C, int P, int NT>
__device__ __forceinline__ void load_tile_f32(float* dst, const float* __restrict__ src, int row0, int nr, int col0,
                                              int nc, int ny, int nx) {
  const bool inner = row0 >= 0 && row0 + nr <= ny && col0 >= 0 && col0 + nc <= nx;
  if (inner && ((col0 | nx | nc) & 1) == 0 && (reinterpret_cast<uintptr_t>(src) & 7) == 0 && (P & 1) == 0) {
    constexpr int C2 = C / 2;
    const int nc2 = nc / 2;
    const float2* s2 = reinterpret_cast<const float2*>(src + (size_t)row0 * nx + col0);
    const size_t pitch2 = (size_t)nx / 2;
    for (int k = threadIdx.x; k < R * C2; k += NT) {
      const int r = k / C2, c = k - r * C2;
      if (r < nr && c < nc2) *reinterpret_cast<float2*>(dst + r * P + 2 * c) = __ldg(s2 + r * pitch2 + c);
    }
    return;
  }
  for (int k = threadIdx.x; k < R * C; k += NT) {
    const int r = k / C, c = k - r * C;
    if (r < nr && c < nc)
      dst[r * P + c] = __ldg(src + (size_t)reflect_index(row0 + r, ny) * nx + reflect_index(col0 + c, nx));
  }
}
template <int R, int C, int P, int NT>
__device__ __forceinline__ void load_tile_f64(float* dst, const double* __restrict__ src, int row0, int nr, int col0,
                                              int nc, int ny, int nx) {
  const bool inner = row0 >= 0 && row0 + nr <= ny && col0 >= 0 && col0 + nc <= nx;
  if (inner && ((col0 | nx | nc) & 1) == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0 && (P & 1) == 0) {
    constexpr int C2 = C / 2;
    const int nc2 = nc / 2;
    const double2* s2 = reinterpret_cast<const double2*>(src + (size_t)row0 * nx + col0);
    const size_t pitch2 = (size_t)nx / 2;
    for (int k = threadIdx.x; k < R * C2; k += NT) {
      const int r = k / C2, c = k - r * C2;
      if (r < nr && c < nc2) {
        const double2 v = __ldg(s2 + r * pitch2 + c);
        *reinterpret_cast<float2*>(dst + r * P + 2 * c) =
            make_float2(f32_of_pos_f64_fast(v.x), f32_of_pos_f64_fast(v.y));
      }
    }
    return;
  }
  for (int k = threadIdx.x; k < R * C; k += NT) {
    const int r = k / C, c = k - r * C;
    if (r < nr && c < nc)
      dst[r * P + c] =
          f32_of_pos_f64_fast(__ldg(src + (size_t)reflect_index(row0 + r, ny) * nx + reflect_index(col0 + c, nx)));
  }
}

}  // namespace part
}  // namespace tf
