// tf_rhs_packed.cuh -- the FP32-bulk residual kernel on packed FP32x2 pipes.
//
// The residual G = u_k + theta dt D(u_k) - b^n of eq. CrankNicolson in
// double-float, with D the flux-form operator of Sec. Flux Discretization,
// or the explicit part b^n = u^n - (1 - theta) dt D(u^n) (the computation of
// k_rhs<ModeF32B>, tf_sweeps.cuh, with fewer FP32 operations).  Each lane
// carries two horizontally adjacent cells through every double-float
// operation, one lane each of the sm_100+ paired FP32 instructions
// (add/mul/fma on float2).  Used for the (n, m) = (3, 2) power law; other
// models take the scalar kernel.
//
// Where the operations are saved:
//   * differences of neighbouring heights.  Where the heights a row step
//     reads (three rows of a strip, halo included) all lie within 25% of
//     each other, the difference of two leading floats is exact (Sterbenz)
//     and so are the sums of up to four of them (they stay below the
//     smallest height's binade), so a height difference is (hi - hi',
//     lo - lo') and the Laplacian's leading part a plain sum; the trailing
//     parts round at 2^-24 of values that are themselves 2^-24 of the
//     heights.  Other row steps take the general double-float operations
//     (TwoSum throughout).
//   * 1/h: the MUFU reciprocal y of the leading float refined by one Newton
//     step in double-float arithmetic, 1/h = y + y (1 - h y), which carries
//     the square of the reciprocal's 2^-23 error.
//   * face fluxes and the divergence stay unnormalised until G is formed.
//   * no shared-memory staging of the film or of intermediate values: a
//     warp keeps its rows in registers and trades neighbours by shuffles.
#pragma once

#include "tf_partition.cuh"

namespace tf {

// ---------------------------------------------------------------------------
// packed double-float: lane-wise the operations of tf_numeric.cuh

struct df2 {
  float2 hi, lo;
};

// (the paired FP32 operations p_add, p_mul, p_fma, ... are in tf_partition.cuh)

__device__ __forceinline__ void p_two_sum(float2 a, float2 b, float2& s, float2& e) {
  s = p_add(a, b);
  const float2 bb = p_sub(s, a);
  e = p_add(p_sub(a, p_sub(s, bb)), p_sub(b, bb));
}
__device__ __forceinline__ void p_fast_two_sum(float2 a, float2 b, float2& s, float2& e) {
  s = p_add(a, b);
  e = p_sub(b, p_sub(s, a));
}
__device__ __forceinline__ df2 d2(float2 hi, float2 lo) {
  df2 r;
  r.hi = hi;
  r.lo = lo;
  return r;
}
__device__ __forceinline__ df2 d2_splat(df64 a) { return d2(p_splat(a.hi), p_splat(a.lo)); }
__device__ __forceinline__ df2 d2_neg(df2 a) { return d2(p_neg(a.hi), p_neg(a.lo)); }
// lazy (unnormalised) add / multiply and the fold: df_add_u, df_mul_u, df_norm
__device__ __forceinline__ df2 d2_add_u(df2 a, df2 b) {
  float2 s, e;
  p_two_sum(a.hi, b.hi, s, e);
  return d2(s, p_add(e, p_add(a.lo, b.lo)));
}
// a - b: the TwoSum of (a.hi, -b.hi) written with subtractions, so that no
// operand is negated on its own ((-b) - bb = -(b + bb) exactly)
__device__ __forceinline__ df2 d2_sub_u(df2 a, df2 b) {
  const float2 s = p_sub(a.hi, b.hi);
  const float2 bb = p_sub(s, a.hi);
  const float2 e = p_sub(p_sub(a.hi, p_sub(s, bb)), p_add(b.hi, bb));
  return d2(s, p_add(e, p_sub(a.lo, b.lo)));
}
// -p exactly (0 - p)
__device__ __forceinline__ float2 p_negz(float2 p) { return p_sub(make_float2(0.0f, 0.0f), p); }
__device__ __forceinline__ df2 d2_mul_u(df2 a, df2 b) {
  const float2 p = p_mul(a.hi, b.hi);
  float2 e = p_fma(a.hi, b.hi, p_neg(p));  // measured cheaper than fma(., ., 0 - p)
  e = p_fma(a.hi, b.lo, e);
  e = p_fma(a.lo, b.hi, e);
  return d2(p, e);
}
__device__ __forceinline__ df2 d2_norm(df2 a) {
  float2 s, e;
  p_fast_two_sum(a.hi, a.lo, s, e);
  return d2(s, e);
}
// normalised add / multiply: operator+ and operator* of df64
__device__ __forceinline__ df2 d2_add(df2 a, df2 b) {
  float2 s, e;
  p_two_sum(a.hi, b.hi, s, e);
  e = p_add(e, p_add(a.lo, b.lo));
  p_fast_two_sum(s, e, s, e);
  return d2(s, e);
}
__device__ __forceinline__ df2 d2_sub(df2 a, df2 b) { return d2_add(a, d2_neg(b)); }
__device__ __forceinline__ df2 d2_mul(df2 a, df2 b) {
  float2 p = p_mul(a.hi, b.hi);
  float2 e = p_fma(a.hi, b.hi, p_negz(p));
  e = p_fma(a.hi, b.lo, e);
  e = p_fma(a.lo, b.hi, e);
  p_fast_two_sum(p, e, p, e);
  return d2(p, e);
}
// 1/a as df_rcp: the correctly rounded float reciprocal (what 1.0f / x
// gives), refined by one double-float Newton step
__device__ __forceinline__ df2 d2_rcp(df2 a) {
  const df2 Y = d2(make_float2(__frcp_rn(a.hi.x), __frcp_rn(a.hi.y)), p_splat(0.0f));
  const df2 r = d2_sub(d2(p_splat(1.0f), p_splat(0.0f)), d2_mul(a, Y));
  return d2_add(Y, d2_mul(Y, r));
}

// ---------------------------------------------------------------------------
// height differences and the reciprocal

// the difference of two double-float heights: exact leading part when the
// two leading floats are within a factor 2 (FAST), else the general one
template <bool FAST> __device__ __forceinline__ df2 hdiff(df2 a, df2 b) {
  if constexpr (FAST) return d2(p_sub(a.hi, b.hi), p_sub(a.lo, b.lo));
  return d2_sub_u(a, b);
}
// 1/a for a positive double-float a (the refined MUFU reciprocal)
__device__ __forceinline__ df2 d2_rcp_fast(df2 a) {
  const float2 y = make_float2(rcp(a.hi.x), rcp(a.hi.y));
  // t = -(1 - a y) exactly: fma(a.hi, y, -1), then fma(a.lo, y, .)
  float2 t = p_fma(a.hi, y, p_splat(-1.0f));
  t = p_fma(a.lo, y, t);
  return d2(y, p_negz(p_mul(y, t)));
}

// ---------------------------------------------------------------------------
// the kernel
//
// Each warp walks a strip of kSW = 60 columns down a segment of rows.  Lane
// l holds the cell pair (x0 - 2 + 2l, x0 - 1 + 2l) of the strip (lanes 0
// and 31 are halo), and the warp carries from one row to the next, in
// registers, the heights of the current and the next row, the current
// row's Laplacian and mobilities and the flux through the face above it.  A
// row step takes one new row of heights, forms the next row's cell values
// (x neighbours by warp shuffles), the face between the two rows, the
// current row's x faces and its G.  A cell's value, a face's flux and G
// are each formed once per strip, from the same operands in the same order
// wherever they are formed.  The choice between the exact and the general
// height differences is made per row step, over the three rows of heights
// that step reads.

// Constants of a launch.  The Laplacian is carried unscaled (the plain sum
// of height differences), so the face fluxes are ds^2 times those of the
// operator: the f1 term takes f1 ds^2 = A1 ds^2 - B1 ds^2 / h, and the
// divergence is scaled by gscale / ds^2.
struct StripK {
  df64 C, A1s, B1s;  // C, A1 ds^2, B1 ds^2
  df64 gs;           // gscale / ds^2 (theta dt or (1 - theta) dt, / (2 ds^4))
  df64 gs2;          // the residual's theta dt / (2 ds^4), for kRhsBoth
  int unitC;         // C == 1
};
TF_HD StripK strip_consts(const ModelK& M, const StepK& K, bool expl) {
  const double ds2 = 1.0 / M.inv_ds2, i4 = 0.5 * M.inv_ds2 * M.inv_ds2;
  StripK k;
  k.C = from_f64<df64>(M.C);
  k.A1s = from_f64<df64>(M.A1 * ds2);
  k.B1s = from_f64<df64>(M.B1 * ds2);
  k.gs = from_f64<df64>(i4 * (expl ? K.expl_dt : K.theta_dt));
  k.gs2 = from_f64<df64>(i4 * K.theta_dt);
  k.unitC = M.C == 1.0;
  return k;
}

constexpr int kSW = 60;  // output columns of a strip
constexpr int kST = 128;  // threads per block
constexpr int kSWarps = kST / 32;


// one row of heights of the lane's pair, as stored (reflected at the walls)
__device__ __forceinline__ double2 strip_load(const double* __restrict__ u, int nx, int ny, int j, int xa,
                                              bool inner) {
  const size_t row = (size_t)((unsigned)j < (unsigned)ny ? j : reflect_index(j, ny)) * nx;
  if (inner) return __ldg(reinterpret_cast<const double2*>(u + row + xa));
  double2 v;
  v.x = __ldg(u + row + reflect_index(xa, nx));
  v.y = __ldg(u + row + reflect_index(xa + 1, nx));
  return v;
}
// the pair as double-float (the leading 24 bits, and the next 29 rounded to
// a float scaled by 2^(e - 1075): the split of df_of_pos_f64_fast, with the
// scaling as a multiply by a power of two), and the warp's range of
// leading-float bits
__device__ __forceinline__ df2 strip_conv(double2 v, unsigned& lo, unsigned& hi) {
  const float ha = f32_of_pos_f64_fast(v.x), hb = f32_of_pos_f64_fast(v.y);
  const unsigned ba = __float_as_uint(ha), bb = __float_as_uint(hb);
  const float ra = __uint2float_rn((unsigned)__double_as_longlong(v.x) & 0x1fffffffu);
  const float rb = __uint2float_rn((unsigned)__double_as_longlong(v.y) & 0x1fffffffu);
  const float2 sc = make_float2(__uint_as_float((ba & 0x7f800000u) - (52u << 23)),
                                __uint_as_float((bb & 0x7f800000u) - (52u << 23)));
  lo = __reduce_min_sync(0xffffffffu, min(ba, bb));
  hi = __reduce_max_sync(0xffffffffu, max(ba, bb));
  return d2(make_float2(ha, hb), p_mul(make_float2(ra, rb), sc));
}
__device__ __forceinline__ bool strip_fast(unsigned lo, unsigned hi) {
  return lo > 0u && hi < 0x7f800000u && __uint_as_float(hi) <= 1.25f * __uint_as_float(lo);
}

// Laplacian (unscaled), f0 and f1 ds^2 of the pair U with the rows above
// (Um) and below (Up); (lh, ll) is the left neighbour's height, (rh, rl) the right one's
template <bool FAST>
__device__ __forceinline__ void strip_cells(const StripK& K, const df2& U, const df2& Um, const df2& Up, float lh,
                                            float ll, float rh, float rl, df2& lap, df2& f0, df2& f1) {
  const df2 E = d2(make_float2(U.hi.y, rh), make_float2(U.lo.y, rl));
  const df2 Wn = d2(make_float2(lh, U.hi.x), make_float2(ll, U.lo.x));
  df2 l;
  if constexpr (FAST) {
    const df2 dE = hdiff<true>(E, U), dW = hdiff<true>(Wn, U);
    const df2 dS = hdiff<true>(Up, U), dN = hdiff<true>(Um, U);
    l = d2(p_add(p_add(dE.hi, dW.hi), p_add(dS.hi, dN.hi)), p_add(p_add(dE.lo, dW.lo), p_add(dS.lo, dN.lo)));
  } else {
    l = d2_add_u(d2_add_u(d2_sub_u(E, U), d2_sub_u(Wn, U)), d2_add_u(d2_sub_u(Up, U), d2_sub_u(Um, U)));
  }
  lap = l;
  const df2 h2 = d2_mul_u(U, U);
  f0 = K.unitC ? d2_mul_u(h2, U) : d2_mul_u(d2_mul_u(d2_splat(K.C), h2), U);
  f1 = d2_sub_u(d2_splat(K.A1s), d2_mul_u(d2_splat(K.B1s), d2_rcp_fast(U)));
}

struct StripState {
  df2 U0, U1;           // heights of rows j, j + 1
  float Lh, Ll;         // left neighbour's height in row j
  df2 lap, f0, f1;      // cell values of row j
  df2 FyM;              // flux through the face between rows j - 1 and j
};

// One row step: from the state at row j and the heights U2 of row j + 2,
// G of row j (when `out`), then the state at row j + 1.  Returns max|G|
// of the lane's cells.
template <int KIND, bool FAST>
__device__ __forceinline__ float strip_step(StripState& s, const df2& U2, const df2& B, bool out, int j, int a,
                                            bool lane_out, const StripK& RK, int nx, int ny,
                                            df64* __restrict__ bn, float* __restrict__ rhs,
                                            float* __restrict__ ulp) {
  constexpr unsigned F = 0xffffffffu;
  // x faces left of the lane's two cells, (a - 1 | a) and (a | a + 1), and
  // the x part of their divergence
  df2 dx = d2(p_splat(0.0f), p_splat(0.0f));
  if (out) {
    const float lph = __shfl_up_sync(F, s.lap.hi.y, 1), lpl = __shfl_up_sync(F, s.lap.lo.y, 1);
    const float f0h = __shfl_up_sync(F, s.f0.hi.y, 1), f0l = __shfl_up_sync(F, s.f0.lo.y, 1);
    const float f1h = __shfl_up_sync(F, s.f1.hi.y, 1), f1l = __shfl_up_sync(F, s.f1.lo.y, 1);
    const df2 f0P = d2(make_float2(f0h, s.f0.hi.x), make_float2(f0l, s.f0.lo.x));
    const df2 f1P = d2(make_float2(f1h, s.f1.hi.x), make_float2(f1l, s.f1.lo.x));
    const df2 lP = d2(make_float2(lph, s.lap.hi.x), make_float2(lpl, s.lap.lo.x));
    const df2 uP = d2(make_float2(s.Lh, s.U0.hi.x), make_float2(s.Ll, s.U0.lo.x));
    df2 Fx = d2_add_u(d2_mul_u(d2_add_u(f0P, s.f0), d2_sub_u(s.lap, lP)),
                      d2_mul_u(d2_add_u(f1P, s.f1), hdiff<FAST>(s.U0, uP)));
    if (!(a - 1 >= 0 && a < nx)) Fx.hi.x = Fx.lo.x = 0.0f;
    if (!(a >= 0 && a + 1 < nx)) Fx.hi.y = Fx.lo.y = 0.0f;
    const float nh = __shfl_down_sync(F, Fx.hi.x, 1), nl = __shfl_down_sync(F, Fx.lo.x, 1);
    dx = d2_sub_u(d2(make_float2(Fx.hi.y, nh), make_float2(Fx.lo.y, nl)), Fx);
  }
  // cell values of row j + 1
  const float l1h = __shfl_up_sync(F, s.U1.hi.y, 1), l1l = __shfl_up_sync(F, s.U1.lo.y, 1);
  const float r1h = __shfl_down_sync(F, s.U1.hi.x, 1), r1l = __shfl_down_sync(F, s.U1.lo.x, 1);
  df2 lap1, f01, f11;
  strip_cells<FAST>(RK, s.U1, s.U0, U2, l1h, l1l, r1h, r1l, lap1, f01, f11);
  // the face between rows j and j + 1 (zero on the walls)
  df2 FyP = d2_add_u(d2_mul_u(d2_add_u(s.f0, f01), d2_sub_u(lap1, s.lap)),
                     d2_mul_u(d2_add_u(s.f1, f11), hdiff<FAST>(s.U1, s.U0)));
  if (!(j >= 0 && j + 1 < ny)) FyP = d2(p_splat(0.0f), p_splat(0.0f));
  float g = 0.0f;
  if (out && lane_out && a < nx) {
    const df2 dp = d2_add_u(dx, d2_sub_u(FyP, s.FyM));
    const df2 uc = s.U0;
    const bool two = a + 1 < nx;
    const size_t idx = (size_t)j * nx + a;
    const df2 gscale = d2_splat(RK.gs);
    if constexpr (KIND == kRhsExplicit) {
      const df2 b = d2_norm(d2_sub_u(uc, d2_mul_u(gscale, dp)));
      bn[idx] = df_make(b.hi.x, b.lo.x);
      if (two) bn[idx + 1] = df_make(b.hi.y, b.lo.y);
    } else {
      df2 bv;
      if constexpr (KIND == kRhsBoth) {
        bv = d2_norm(d2_sub_u(uc, d2_mul_u(gscale, dp)));
        bn[idx] = df_make(bv.hi.x, bv.lo.x);
        if (two) bn[idx + 1] = df_make(bv.hi.y, bv.lo.y);
        if (!two) bv = d2(make_float2(bv.hi.x, 1.0f), make_float2(bv.lo.x, 0.0f));  // as the loaded pair
      } else {
        bv = B;
      }
      const df2 gs = KIND == kRhsBoth ? d2_splat(RK.gs2) : gscale;
      // -G = (b^n - u) - gs dp: the negation of G's operations, exactly
      const df2 Gn = d2_norm(d2_sub_u(d2_sub_u(bv, uc), d2_mul_u(gs, dp)));
      const float2 gl = p_add(Gn.hi, Gn.lo);
      // FP32 film for the sweeps: the leading float of the double-float height
      if (two && ((nx | a) & 1) == 0) {
        *reinterpret_cast<float2*>(rhs + idx) = gl;
        *reinterpret_cast<float2*>(ulp + idx) = uc.hi;
      } else {
        rhs[idx] = gl.x;
        ulp[idx] = uc.hi.x;
        if (two) {
          rhs[idx + 1] = gl.y;
          ulp[idx + 1] = uc.hi.y;
        }
      }
      g = fabsf(gl.x);
      const float ag = two ? fabsf(gl.y) : 0.0f;
      if (!(ag <= g)) g = ag;
    }
  }
  s.U0 = s.U1;
  s.U1 = U2;
  s.Lh = l1h;
  s.Ll = l1l;
  s.lap = lap1;
  s.f0 = f01;
  s.f1 = f11;
  s.FyM = FyP;
  return g;
}

// Rows reach the warps through shared memory: each warp has a ring of four
// rows of heights and four of b^n, filled with asynchronous copies two rows
// ahead of their use, so no register holds a load in flight.
struct StripRing {
  double2 u[4][32];  // the lane's pair of heights
  float4 b[4][32];   // the lane's pair of b^n (hi, lo, hi, lo)
};

// queue the copy of row j of heights into dst (reflected at the walls)
__device__ __forceinline__ void strip_copy_u(double2* dst, const double* __restrict__ u, int nx, int ny, int j,
                                             int xa, bool inner) {
  const double* row = u + (size_t)((unsigned)j < (unsigned)ny ? j : reflect_index(j, ny)) * nx;
  if (inner) {
    __pipeline_memcpy_async(dst, row + xa, 16);
  } else {
    __pipeline_memcpy_async(reinterpret_cast<double*>(dst), row + reflect_index(xa, nx), 8);
    __pipeline_memcpy_async(reinterpret_cast<double*>(dst) + 1, row + reflect_index(xa + 1, nx), 8);
  }
}
// queue the copy of the lane's b^n of row j (nothing where there is no cell)
__device__ __forceinline__ void strip_copy_bn(float4* dst, const df64* __restrict__ bn, int nx, int ny, int j,
                                              int a, bool lane_out) {
  if (!(lane_out && j < ny && a < nx)) return;
  const size_t idx = (size_t)j * nx + a;
  if (a + 1 < nx && ((nx | a) & 1) == 0) {
    __pipeline_memcpy_async(dst, bn + idx, 16);
  } else {
    __pipeline_memcpy_async(reinterpret_cast<df64*>(dst), bn + idx, 8);
    if (a + 1 < nx) __pipeline_memcpy_async(reinterpret_cast<df64*>(dst) + 1, bn + idx + 1, 8);
  }
}

// KIND: kRhsResidual (G from u_k and the stored b^n), kRhsExplicit (b^n from
// u^n) or kRhsBoth (b^n from u^n, stored, and G of the first iteration,
// u_0 = u^n, from the same stored b^n -- what kRhsResidual would compute).
// Warp w of the grid takes strip w % nstrip and rows [seg_rows * (w /
// nstrip), + seg_rows); one partial result (max|G|) per block.
// DEV (the ensemble graphs): the step's constants *RKd and the grid *ud come
// from device memory; otherwise RKp and up.
template <int KIND, bool DEV = false>
__global__ void __launch_bounds__(kST, 5)
    k_rhs_strip(ModelK M, StripK RKp, const double* __restrict__ up, df64* __restrict__ bn,
                float* __restrict__ rhs, float* __restrict__ ulp, PartX* __restrict__ part, int nstrip,
                int seg_rows, const StripK* __restrict__ RKd = nullptr, const double* const* __restrict__ ud = nullptr) {
  const StripK& RK = DEV ? *RKd : RKp;
  const double* __restrict__ u = DEV ? *ud : up;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nx = M.nx, ny = M.ny;
  const int w = blockIdx.x * kSWarps + warp;
  const int nseg = (ny + seg_rows - 1) / seg_rows;
  __shared__ StripRing ring[kSWarps];
  float g = 0.0f;
  if (w < nstrip * nseg) {
    const int x0 = (w % nstrip) * kSW, ja = (w / nstrip) * seg_rows;
    const int jb = min(ja + seg_rows, ny);
    const int a = x0 - 2 + 2 * lane;  // the lane's first cell
    const bool lane_out = lane >= 1 && lane <= kSW / 2;
    const bool inner = x0 - 2 >= 0 && x0 + kSW + 2 <= nx && (nx & 1) == 0 &&
                       (reinterpret_cast<uintptr_t>(u) & 15) == 0;
    StripRing& R = ring[warp];
    // rows ja - 2 .. ja directly; rows ja + 1, ja + 2 (and b^n of rows ja,
    // ja + 1) queued
    unsigned lo0, hi0, lo1, hi1, lo2, hi2, lo3, hi3;
    const df2 Um2 = strip_conv(strip_load(u, nx, ny, ja - 2, a, inner), lo0, hi0);
    const df2 Um1 = strip_conv(strip_load(u, nx, ny, ja - 1, a, inner), lo1, hi1);
    const df2 Ua = strip_conv(strip_load(u, nx, ny, ja, a, inner), lo2, hi2);
    for (int q = 1; q <= 2; ++q) {
      strip_copy_u(&R.u[(ja + q) & 3][lane], u, nx, ny, ja + q, a, inner);
      if constexpr (KIND == kRhsResidual) strip_copy_bn(&R.b[(ja + q - 1) & 3][lane], bn, nx, ny, ja + q - 1, a, lane_out);
      __pipeline_commit();
    }
    StripState s;
    s.U0 = Um1;
    s.U1 = Ua;
    s.FyM = d2(p_splat(0.0f), p_splat(0.0f));
    {  // cell values of row ja - 1
      constexpr unsigned F = 0xffffffffu;
      const float lh = __shfl_up_sync(F, Um1.hi.y, 1), ll = __shfl_up_sync(F, Um1.lo.y, 1);
      const float rh = __shfl_down_sync(F, Um1.hi.x, 1), rl = __shfl_down_sync(F, Um1.lo.x, 1);
      s.Lh = lh;
      s.Ll = ll;
      if (strip_fast(min(lo0, min(lo1, lo2)), max(hi0, max(hi1, hi2))))
        strip_cells<true>(RK, Um1, Um2, Ua, lh, ll, rh, rl, s.lap, s.f0, s.f1);
      else
        strip_cells<false>(RK, Um1, Um2, Ua, lh, ll, rh, rl, s.lap, s.f0, s.f1);
    }
    // row steps j = ja - 1 (state only) .. jb - 1; the state's rows j, j + 1
    // have ranges (lo1, hi1), (lo2, hi2).  Step j queues heights of row
    // j + 4 and b^n of row j + 3 (slots last read two steps before) and
    // waits for the copies of step j - 2 (heights j + 2, b^n j + 1).
    for (int j = ja - 1; j < jb; ++j) {
      const bool out = j >= ja;
      strip_copy_u(&R.u[(j + 4) & 3][lane], u, nx, ny, j + 4, a, inner);
      if constexpr (KIND == kRhsResidual) strip_copy_bn(&R.b[(j + 3) & 3][lane], bn, nx, ny, j + 3, a, lane_out);
      __pipeline_commit();
      __pipeline_wait_prior(2);
      df2 B = d2(p_splat(1.0f), p_splat(0.0f));
      if constexpr (KIND == kRhsResidual) {
        if (out) {
          const float4 v = R.b[j & 3][lane];
          B = d2(make_float2(v.x, v.z), make_float2(v.y, v.w));
        }
      }
      const df2 U2 = strip_conv(R.u[(j + 2) & 3][lane], lo3, hi3);
      float gj;
      if (strip_fast(min(lo1, min(lo2, lo3)), max(hi1, max(hi2, hi3))))
        gj = strip_step<KIND, true>(s, U2, B, out, j, a, lane_out, RK, nx, ny, bn, rhs, ulp);
      else
        gj = strip_step<KIND, false>(s, U2, B, out, j, a, lane_out, RK, nx, ny, bn, rhs, ulp);
      if (!(gj <= g)) g = gj;
      lo1 = lo2;
      hi1 = hi2;
      lo2 = lo3;
      hi2 = hi3;
    }
    __pipeline_wait_prior(0);  // no copy outlives the warp
  }
  if constexpr (KIND == kRhsExplicit) return;
  for (int o = 16; o > 0; o >>= 1) {
    const float g2 = __shfl_xor_sync(0xffffffffu, g, o);
    if (!(g2 <= g)) g = g2;
  }
  __shared__ float red[kSWarps];
  if (lane == 0) red[warp] = g;
  __syncthreads();
  if (threadIdx.x == 0) {
    float mx = red[0];
    for (int k = 1; k < kSWarps; ++k)
      if (!(red[k] <= mx)) mx = red[k];
    PartX p;
    p.gnorm = (double)mx;
    p.pivot = 0;
    p.pad = 0;
    part[blockIdx.x] = p;
  }
}

}  // namespace tf
