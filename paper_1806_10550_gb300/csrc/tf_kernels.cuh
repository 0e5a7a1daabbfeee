// tf_kernels.cuh -- CUDA kernels of the Newton--ADI thin-film time step.
//
// One templated kernel set serves both precision modes (Mode = ModeFP64 or
// ModeF32B, see tf_numeric.cuh for the double-float arithmetic):
//   HP  precision of the explicit part b^n, the residual G and the update;
//   LP  precision of the Jacobian assembly and the pentadiagonal solves.
//
// Discretisation (Lam, Cummings & Kondic):
//   Lap_c  = sum over existing neighbours nb of (u_nb - u_c) / ds^2
//            (five points; a wall neighbour is the cell itself: even
//            reflection, eq. BoundaryConditions)
//   F(p,q) = fbar0 (Lap_q - Lap_p)/ds + fbar1 (u_q - u_p)/ds through each
//            interior face, fbar = mean of the two cell values (Sec. Flux
//            Discretization); wall faces carry no flux
//   D_c    = [F_east - F_west + F_north - F_south] / ds     (eq. GovEqnCell2)
//   b^n    = u^n - (1-theta) dt D(u^n);  G(u_k) = u_k + theta dt D(u_k) - b^n
//   J_x    = d(x-face fluxes)/du without the derivative through the y part
//            of the Laplacian (the neglected mixed term of eq.
//            DirectionSplit); J_y likewise.
//   (I + theta dt J_x) w = -G on rows, (I + theta dt J_y) v = w on columns,
//   u_{k+1} = u_k + v                                (eqs. JacobianSystem1-3)
// The line solves themselves live in tf_sweeps.cuh (residual kernel and
// shared line machinery) and tf_line_sweeps.cuh (the x and y sweeps).
#pragma once

#include <cuda_runtime.h>

#include "tf_numeric.cuh"

namespace tf {

// ---------------------------------------------------------------------------
// constants

struct ModelK {
  int nx, ny;
  int model;  // 0 power law, 1 linear, 2 NLC, 3 polymer
  int n, m;
  double inv_ds, inv_ds2, inv_ds3;
  double C;       // f0 = C h^3
  double A1, B1;  // f1 = A1 s^(m-2) - B1 s^(n-2), s = 1/h
  double c0, c1;  // linear model
  double b;       // precursor scale of the NLC Pi
  double nlc_K, nlc_N, nlc_beta, nlc_w;
  double pol_C, pol_A1, pol_A2, pol_d;  // A1 = A_SiOx, A2 = A_Si
};

struct StepK {
  double theta_dt;  // theta dt
  double expl_dt;   // (1 - theta) dt
};

struct PartX {  // per-block partial results of the x pass
  double gnorm;
  int pivot;
  int pad;
};
// Exact sums of the 2^-36 fixed-point images of grid values (the mass
// diagnostic): a 128-bit unsigned integer as two 64-bit words, so no grid
// the library accepts (fewer than 2^31 cells, each image below 2^63) can
// overflow it, and the sum does not depend on the order of the additions.
struct Mass128 {
  unsigned long long lo, hi;
};
TF_HD void mass_add(Mass128& a, unsigned long long v) {
  a.lo += v;
  a.hi += a.lo < v ? 1ull : 0ull;
}
TF_HD void mass_add(Mass128& a, const Mass128& b) {
  a.lo += b.lo;
  a.hi += b.hi + (a.lo < b.lo ? 1ull : 0ull);
}
// The sum as a double (the value times 2^-36), converted once at the end.
inline double mass_value(const Mass128& m) {
  return m.hi ? ldexp((double)m.hi, 28) + ldexp((double)m.lo, -36) : ldexp((double)m.lo, -36);
}

struct PartY {  // per-block partial results of the y pass
  double err, hmin;
  Mass128 mass;
  int nonfinite, pivot;
};
struct Scalars {
  double err, gnorm, hmin;
  Mass128 mass;  // exact sum of the 2^-36 fixed-point images of the grid values
  int nonfinite, pivot;
};

struct ModeFP64 {
  typedef double HP;
  typedef double LP;
  static constexpr int kSweepBlocks = 1;  // sweep blocks per SM (shared memory)
};
struct ModeF32B {
  typedef df64 HP;
  typedef float LP;
  static constexpr int kSweepBlocks = 2;
};

// ---------------------------------------------------------------------------
// precision helpers

template <class T> TF_HD T from_f64(double d);
template <> TF_HD double from_f64<double>(double d) { return d; }
template <> TF_HD df64 from_f64<df64>(double d) { return df_of_f64(d); }
template <> TF_HD float from_f64<float>(double d) { return f32_trunc_of_f64(d); }

template <class LP, class HP> TF_HD LP to_lp(HP x);
template <> TF_HD double to_lp<double, double>(double x) { return x; }
template <> TF_HD float to_lp<float, df64>(df64 x) { return x.hi + x.lo; }

TF_HD double to_f64(double x) { return x; }
TF_HD double to_f64(df64 x) { return f64_of_df(x); }
TF_HD double to_f64(float x) { return f64_of_f32(x); }

TF_HD double rcp(double x) { return 1.0 / x; }
TF_HD float rcp(float x) {
#ifdef __CUDA_ARCH__
  float r;  // the MUFU reciprocal alone, about 1 ulp: FP32 Jacobian and solves only
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
#else
  return 1.0f / x;
#endif
}
TF_HD df64 rcp(df64 x) { return df_rcp(x); }

template <class T> TF_HD T one();
template <> TF_HD double one<double>() { return 1.0; }
template <> TF_HD float one<float>() { return 1.0f; }
template <> TF_HD df64 one<df64>() { return df_make(1.0f, 0.0f); }
template <class T> TF_HD T zero();
template <> TF_HD double zero<double>() { return 0.0; }
template <> TF_HD float zero<float>() { return 0.0f; }
template <> TF_HD df64 zero<df64>() { return df_make(0.0f, 0.0f); }

template <class T> TF_HD T ipow(T x, int k) {
  T r = x;
  for (int i = 1; i < k; ++i) r = r * x;
  return r;
}
// h^(-k) written through s = 1/h for k >= 0 and through h for k < 0.
template <class T> TF_HD T hpow_neg(const T& h, const T& s, int k) {
  if (k > 0) return ipow(s, k);
  if (k < 0) return ipow(h, -k);
  return one<T>();
}

template <class T> struct MobC {
  T C, A1, B1, c0, c1, three, half;
  T dA1, dB1;  // (m-2) A1 and (n-2) B1
  int model, n, m;
  bool unitC;  // C == 1
  bool pl32;   // power law with (n, m) = (3, 2)
  // NLC and polymer parameters (evaluated out of line, see pi_model)
  double Cd, b, K, N, beta2, w, pC, pA1, pA12, pd;
};
template <class T> TF_HD MobC<T> mob_consts(const ModelK& M) {
  MobC<T> c;
  c.C = from_f64<T>(M.C);
  c.A1 = from_f64<T>(M.A1);
  c.B1 = from_f64<T>(M.B1);
  c.c0 = from_f64<T>(M.c0);
  c.c1 = from_f64<T>(M.c1);
  c.three = from_f64<T>(3.0);
  c.half = from_f64<T>(0.5);
  c.dA1 = from_f64<T>((double)(M.m - 2) * M.A1);
  c.dB1 = from_f64<T>((double)(M.n - 2) * M.B1);
  c.model = M.model;
  c.n = M.n;
  c.m = M.m;
  c.unitC = M.C == 1.0;
  c.pl32 = M.model == 0 && M.n == 3 && M.m == 2;
  c.Cd = M.C;
  c.b = M.b;
  c.K = M.nlc_K;
  c.N = M.nlc_N;
  c.beta2 = M.nlc_beta * M.nlc_beta;
  c.w = M.nlc_w;
  c.pC = M.pol_C;
  c.pA1 = M.pol_A1;
  c.pA12 = M.pol_A1 - M.pol_A2;
  c.pd = M.pol_d;
  return c;
}

// Per-launch constants of the line sweeps and of the residual, converted once
// on the host: kernels read them from the parameter space and never convert
// or recompute them per cell.
template <class T> struct LineK {
  MobC<T> ml;
  T inv_ds2;  // 1/ds^2
  T k3, k1;   // theta dt/(2 ds^4) and theta dt/(2 ds^2): the band's face scales
  // folded factors of the (n, m) = (3, 2) power law (ml.pl32):
  // F0 = k3 C h^3, F1 = k1 A1 - k1 B1 / h, D0 = (k1 / ds^2) 3 C h^2 (the
  // Laplacian left unscaled), D1 = k1 B1 / h^2
  T pF0, pF1a, pF1b, pD0, pD1;
};
template <class T> TF_HD LineK<T> line_consts(const ModelK& M, const StepK& K) {
  LineK<T> L;
  L.ml = mob_consts<T>(M);
  L.inv_ds2 = (T)M.inv_ds2;
  const double k3 = 0.5 * K.theta_dt * M.inv_ds3 * M.inv_ds, k1 = 0.5 * K.theta_dt * M.inv_ds2;
  L.k3 = (T)k3;
  L.k1 = (T)k1;
  L.pF0 = (T)(k3 * M.C);
  L.pF1a = (T)(k1 * M.A1);
  L.pF1b = (T)(k1 * M.B1);
  L.pD0 = (T)(k1 * M.inv_ds2 * 3.0 * M.C);
  L.pD1 = (T)(k1 * M.B1);
  return L;
}
// What a residual-stencil kernel forms: the residual of an iteration, the
// explicit part of a step, or both from one D(u^n) (a step's first
// iteration starts from u_0 = u^n).
enum { kRhsResidual = 0, kRhsExplicit = 1, kRhsBoth = 2 };

template <class T> struct RhsK {
  MobC<T> mc;
  T inv_ds2, four;
  T gscale;   // theta dt/(2 ds^2), or (1 - theta) dt/(2 ds^2) for the explicit part
  T gscale2;  // theta dt/(2 ds^2) (the residual's, when one kernel forms both)
};
// gscale: theta dt/(2 ds^2) for the residual, (1 - theta) dt/(2 ds^2) for
// the explicit part (expl); gscale2 always the residual's.
template <class T> inline RhsK<T> rhs_consts(const ModelK& M, const StepK& K, bool expl = false) {
  RhsK<T> R;
  R.mc = mob_consts<T>(M);
  R.inv_ds2 = from_f64<T>(M.inv_ds2);
  R.four = from_f64<T>(4.0);
  R.gscale = from_f64<T>(0.5 * M.inv_ds2 * (expl ? K.expl_dt : K.theta_dt));
  R.gscale2 = from_f64<T>(0.5 * M.inv_ds2 * K.theta_dt);
  return R;
}

template <class T> struct MobPair {
  T a, b;
};

// Pi', Pi'' of the NLC and polymer models (Sec. Thin Film Models), in R =
// float (the FP32 Jacobian) or double (everything FP64-class):
//   NLC (eqs. DisjPressNLC, mh_model): Pi = K[r^3 - r^2] + (N/2) q^2, r = b/h,
//     q = m(h)/h = g h/D, D = h^2 + beta^2, g = [1 + tanh((h - 2b)/w)]/2;
//     Pi' = K(2r^2 - 3r^3)/h + N q q',  Pi'' = K(12r^3 - 6r^2)/h^2 + N(q'^2 + q q''),
//     q' = g' h/D + g(beta^2 - h^2)/D^2,
//     q'' = g'' h/D + 2g'(beta^2 - h^2)/D^2 + 2g h(h^2 - 3beta^2)/D^3,
//     g' = (1 - t^2)/(2w), g'' = -t(1 - t^2)/w^2, t = tanh((h - 2b)/w).
//   Polymer (eq. DisjPressPolymer), Pi = -psi':
//     Pi' = -72 Cp/h^10 + A1/(2 pi h^4) - (A1 - A2)/(2 pi (h + d)^4),
//     Pi'' = 720 Cp/h^11 - 2A1/(pi h^5) + 2(A1 - A2)/(pi (h + d)^5).
__host__ __device__ inline float r_tanh(float x) { return tanhf(x); }
__host__ __device__ inline double r_tanh(double x) { return tanh(x); }
template <class R, class T>
__host__ __device__ inline void pi_model(const MobC<T>& c, R h, R& d1, R& d2) {
  const R ih = R(1) / h;
  if (c.model == 3) {
    const R pi = R(3.14159265358979323846);
    const R Cp = R(c.pC), A1 = R(c.pA1), A12 = R(c.pA12), ie = R(1) / (h + R(c.pd));
    const R i2 = ih * ih, i4 = i2 * i2, i5 = i4 * ih, i10 = i5 * i5, e2 = ie * ie, e4 = e2 * e2;
    const R k = R(1) / (R(2) * pi);
    d1 = R(-72) * Cp * i10 + k * (A1 * i4 - A12 * e4);
    d2 = R(720) * Cp * i10 * ih - R(4) * k * (A1 * i5 - A12 * e4 * ie);
    return;
  }
  const R b = R(c.b), K = R(c.K), N = R(c.N), be2 = R(c.beta2), iw = R(1) / R(c.w);
  const R r = b * ih, r2 = r * r, r3 = r2 * r;
  const R t = r_tanh((h - R(2) * b) * iw), sech2 = R(1) - t * t;
  const R g = R(0.5) * (R(1) + t), dg = R(0.5) * sech2 * iw, d2g = -t * sech2 * iw * iw;
  const R iD = R(1) / (h * h + be2), bmh = be2 - h * h;
  const R q = g * h * iD;
  const R dq = (dg * h + g * bmh * iD) * iD;
  const R d2q = (d2g * h + (R(2) * dg * bmh + g * R(2) * h * (h * h - R(3) * be2) * iD) * iD) * iD;
  d1 = K * (R(2) * r2 - R(3) * r3) * ih + N * q * dq;
  d2 = K * (R(12) * r3 - R(6) * r2) * ih * ih + N * (dq * dq + q * d2q);
}
// Height and values between T and the arithmetic R of pi_model: float stays
// float; double and double-float evaluate in double.
template <class T> struct PiArith {
  typedef double R;
};
template <> struct PiArith<float> {
  typedef float R;
};
__host__ __device__ inline double to_r(double x) { return x; }
__host__ __device__ inline float to_r(float x) { return x; }
__host__ __device__ inline double to_r(df64 x) { return f64_of_df(x); }
template <class T> __host__ __device__ inline T from_r(typename PiArith<T>::R x);
template <> __host__ __device__ inline double from_r<double>(double x) { return x; }
template <> __host__ __device__ inline float from_r<float>(float x) { return x; }
template <> __host__ __device__ inline df64 from_r<df64>(double x) { return df_of_f64(x); }

// f0 = C h^3 and f1 = h^3 Pi'(h) = A1 h^(2-m) - B1 h^(2-n)
// (Sec. Thin Film Models, eq. GeneralDisPreForm); the linear model has
// constant f0 = c0, f1 = c1.  General exponents and the linear model are
// evaluated out of line, so that kernels inline only the (n, m) = (3, 2)
// power law.
template <class T>
__host__ __device__ __noinline__ MobPair<T> mobility_general(const MobC<T> c, const T h, const T s) {
  MobPair<T> r;
  if (c.model == 1) {
    r.a = c.c0;
    r.b = c.c1;
    return r;
  }
  if (c.model >= 2) {  // NLC, polymer: f0 = C h^3, f1 = h^3 Pi'
    typedef typename PiArith<T>::R R;
    const R hr = to_r(h), h3 = hr * hr * hr;
    R d1, d2;
    pi_model<R>(c, hr, d1, d2);
    r.a = from_r<T>(R(c.Cd) * h3);
    r.b = from_r<T>(h3 * d1);
    return r;
  }
  r.a = c.unitC ? (h * h) * h : c.C * (h * h) * h;
  T a = c.m == 2 ? c.A1 : c.A1 * hpow_neg(h, s, c.m - 2);
  T b = c.n == 2 ? c.B1 : c.B1 * hpow_neg(h, s, c.n - 2);
  r.b = a - b;
  return r;
}
// f0' = 3 C h^2, f1' = -(m-2) A1 h^(1-m) + (n-2) B1 h^(1-n).
template <class T>
__host__ __device__ __noinline__ MobPair<T> mobility_d_general(const MobC<T> c, const T h, const T s) {
  MobPair<T> r;
  if (c.model == 1) {
    r.a = zero<T>();
    r.b = zero<T>();
    return r;
  }
  if (c.model >= 2) {  // f0' = 3 C h^2, f1' = 3 h^2 Pi' + h^3 Pi''
    typedef typename PiArith<T>::R R;
    const R hr = to_r(h), h2 = hr * hr;
    R d1, d2;
    pi_model<R>(c, hr, d1, d2);
    r.a = from_r<T>(R(3) * R(c.Cd) * h2);
    r.b = from_r<T>(R(3) * h2 * d1 + h2 * hr * d2);
    return r;
  }
  r.a = c.three * c.C * (h * h);
  T b = c.dB1 * hpow_neg(h, s, c.n - 1);
  r.b = c.m == 2 ? b : b - c.dA1 * hpow_neg(h, s, c.m - 1);
  return r;
}

// f0, f1, f0', f1' of the NLC and polymer models in one out-of-line call.
template <class T> struct MobQuad {
  T f0, f1, d0, d1;
};
template <class T>
__host__ __device__ __noinline__ MobQuad<T> mobility_model_all(const MobC<T> c, const T h) {
  typedef typename PiArith<T>::R R;
  const R hr = to_r(h), h2 = hr * hr, h3 = h2 * hr;
  R d1, d2;
  pi_model<R>(c, hr, d1, d2);
  MobQuad<T> q;
  q.f0 = from_r<T>(R(c.Cd) * h3);
  q.f1 = from_r<T>(h3 * d1);
  q.d0 = from_r<T>(R(3) * R(c.Cd) * h2);
  q.d1 = from_r<T>(R(3) * h2 * d1 + h3 * d2);
  return q;
}

template <class T>
TF_HD void mobility(const MobC<T>& c, const T& h, const T& s, T& f0, T& f1) {
  if (c.pl32) {  // f1 = A1 - B1 / h
    f0 = c.unitC ? (h * h) * h : c.C * (h * h) * h;
    f1 = c.A1 - c.B1 * s;
    return;
  }
  const MobPair<T> r = mobility_general(c, h, s);
  f0 = r.a;
  f1 = r.b;
}
// f0, f1 and their derivatives together (one evaluation of Pi for the NLC
// and polymer models).
template <class T>
TF_HD void mobility_all(const MobC<T>& c, const T& h, const T& s, T& f0, T& f1, T& d0, T& d1) {
  if (c.model >= 2) {
    const MobQuad<T> q = mobility_model_all(c, h);
    f0 = q.f0;
    f1 = q.f1;
    d0 = q.d0;
    d1 = q.d1;
    return;
  }
  mobility(c, h, s, f0, f1);
  mobility_d(c, h, s, d0, d1);
}

template <class T>
TF_HD void mobility_d(const MobC<T>& c, const T& h, const T& s, T& d0, T& d1) {
  if (c.pl32) {  // f1' = B1 / h^2
    d0 = c.three * c.C * (h * h);
    d1 = c.dB1 * (s * s);
    return;
  }
  const MobPair<T> r = mobility_d_general(c, h, s);
  d0 = r.a;
  d1 = r.b;
}

TF_HD int reflect_index(int i, int n) {
  // Even reflection about the walls: -1 -> 0, -2 -> 1, n -> n-1, n+1 -> n-2
  // (repeated for lines shorter than two cells).
  for (int k = 0; k < 3; ++k) {
    if (i < 0) i = -1 - i;
    if (i >= n) i = 2 * n - 1 - i;
  }
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// ---------------------------------------------------------------------------
// Tile stencil: per-cell quantities, face fluxes and D' on a TR x TC tile
// of cells whose first cell is (j0, x0).  D = (1/2) inv_ds^2 D'.

template <class HP, int TR, int TC> struct StencilSmem {
  HP u[TR + 4][TC + 4];              // u on rows j0-2.., cols x0-2..
  HP lap[TR + 2][TC + 2];            // on rows j0-1.., cols x0-1..
  HP f0[TR + 2][TC + 2], f1[TR + 2][TC + 2], s[TR + 2][TC + 2];
  HP fx[TR][TC + 1];                 // face between cols x0-1+c and x0+c
  HP fy[TR + 1][TC];                 // face between rows j0-1+r and j0+r
};

template <class HP, int TR, int TC>
__device__ __forceinline__ void stencil_load(StencilSmem<HP, TR, TC>& S, const double* __restrict__ u,
                                             const ModelK& M, int j0, int x0, int tid, int nt) {
  for (int k = tid; k < (TR + 4) * (TC + 4); k += nt) {
    int r = k / (TC + 4), c = k - r * (TC + 4);
    int gj = reflect_index(j0 - 2 + r, M.ny), gi = reflect_index(x0 - 2 + c, M.nx);
    S.u[r][c] = from_f64<HP>(__ldg(u + (size_t)gj * M.nx + gi));
  }
}

template <class HP, int TR, int TC>
__device__ __forceinline__ void stencil_cells(StencilSmem<HP, TR, TC>& S, const MobC<HP>& mc,
                                              const HP& inv_ds2, int tid, int nt) {
  for (int k = tid; k < (TR + 2) * (TC + 2); k += nt) {
    int r = k / (TC + 2), c = k - r * (TC + 2);
    HP uc = S.u[r + 1][c + 1];
    HP d = ((S.u[r + 1][c + 2] - uc) + (S.u[r + 1][c] - uc)) +
           ((S.u[r + 2][c + 1] - uc) + (S.u[r][c + 1] - uc));
    S.lap[r][c] = d * inv_ds2;
    HP s = rcp(uc);
    HP f0, f1;
    mobility(mc, uc, s, f0, f1);
    S.s[r][c] = s;
    S.f0[r][c] = f0;
    S.f1[r][c] = f1;
  }
}

// Unscaled face flux F' = (f0p + f0q)(Lq - Lp) + (f1p + f1q)(uq - up);
// F = F' / (2 ds).  Zero through the walls.
template <class HP, int TR, int TC>
__device__ __forceinline__ void stencil_faces(StencilSmem<HP, TR, TC>& S, const ModelK& M, int j0,
                                              int x0, int tid, int nt) {
  for (int k = tid; k < TR * (TC + 1); k += nt) {
    int r = k / (TC + 1), c = k - r * (TC + 1);
    int gp = x0 - 1 + c;  // left cell of the face
    HP F = zero<HP>();
    if (gp >= 0 && gp + 1 < M.nx) {
      int rr = r + 1;  // region row of cell row j0 + r
      F = (S.f0[rr][c] + S.f0[rr][c + 1]) * (S.lap[rr][c + 1] - S.lap[rr][c]) +
          (S.f1[rr][c] + S.f1[rr][c + 1]) * (S.u[rr + 1][c + 2] - S.u[rr + 1][c + 1]);
    }
    S.fx[r][c] = F;
  }
  for (int k = tid; k < (TR + 1) * TC; k += nt) {
    int r = k / TC, c = k - r * TC;
    int gp = j0 - 1 + r;  // lower cell of the face
    HP F = zero<HP>();
    if (gp >= 0 && gp + 1 < M.ny) {
      int cc = c + 1;  // region col of cell col x0 + c
      F = (S.f0[r][cc] + S.f0[r + 1][cc]) * (S.lap[r + 1][cc] - S.lap[r][cc]) +
          (S.f1[r][cc] + S.f1[r + 1][cc]) * (S.u[r + 2][cc + 1] - S.u[r + 1][cc + 1]);
    }
    S.fy[r][c] = F;
  }
}

template <class HP, int TR, int TC>
__device__ __forceinline__ HP stencil_dprime(const StencilSmem<HP, TR, TC>& S, int r, int c) {
  return (S.fx[r][c + 1] - S.fx[r][c]) + (S.fy[r + 1][c] - S.fy[r][c]);
}

// ---------------------------------------------------------------------------
// 2-D stencil kernel: explicit part b^n (OUT_B) or residual G (OUT_G).

template <class Mode, int OUT_G>
__global__ void __launch_bounds__(256)
    k_stencil(ModelK M, StepK K, const double* __restrict__ u, typename Mode::HP* __restrict__ bn,
              double* __restrict__ G, PartX* __restrict__ part) {
  typedef typename Mode::HP HP;
  constexpr int T = 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  StencilSmem<HP, T, T>& S = *reinterpret_cast<StencilSmem<HP, T, T>*>(smem_raw);
  const int tid = threadIdx.y * T + threadIdx.x, nt = T * T;
  const int x0 = blockIdx.x * T, j0 = blockIdx.y * T;
  const MobC<HP> mc = mob_consts<HP>(M);
  const HP inv_ds2 = from_f64<HP>(M.inv_ds2);
  stencil_load(S, u, M, j0, x0, tid, nt);
  __syncthreads();
  stencil_cells(S, mc, inv_ds2, tid, nt);
  __syncthreads();
  stencil_faces(S, M, j0, x0, tid, nt);
  __syncthreads();
  const int r = threadIdx.y, c = threadIdx.x;
  const int gj = j0 + r, gi = x0 + c;
  double g = 0.0;
  if (gj < M.ny && gi < M.nx) {
    const size_t idx = (size_t)gj * M.nx + gi;
    HP dp = stencil_dprime(S, r, c);
    HP uc = S.u[r + 2][c + 2];
    if (OUT_G) {
      HP scale = from_f64<HP>(0.5 * M.inv_ds2 * K.theta_dt);
      HP Gv = (uc - bn[idx]) + scale * dp;
      G[idx] = to_f64(Gv);
      g = fabs(to_f64(Gv));
    } else {
      HP scale = from_f64<HP>(0.5 * M.inv_ds2 * K.expl_dt);
      bn[idx] = uc - scale * dp;
    }
  }
  if (OUT_G) {
    for (int o = 16; o > 0; o >>= 1) g = fmax(g, __shfl_xor_sync(0xffffffffu, g, o));
    __shared__ double red[8];
    if ((tid & 31) == 0) red[tid >> 5] = g;
    __syncthreads();
    if (tid == 0) {
      double mx = red[0];
      for (int k = 1; k < 8; ++k) mx = fmax(mx, red[k]);
      part[blockIdx.y * gridDim.x + blockIdx.x].gnorm = mx;
      part[blockIdx.y * gridDim.x + blockIdx.x].pivot = 0;
    }
  }
}

// ---------------------------------------------------------------------------
// Line band assembly and LU

template <class LP> struct CellLP {
  LP u, lap, f0, f1, d0, d1;
};

// dF of one interior face between line cells p and q = p+1, scaled by
// sc = theta dt / ds, for the columns p-1, p, q, q+1.  pl: p has a left
// neighbour; qr: q has a right neighbour.
template <class LP>
__device__ __forceinline__ void face_dF(const CellLP<LP>& P, const CellLP<LP>& Q, bool pl, bool qr,
                                        LP inv_ds, LP inv_ds3, LP sc, LP dF[4]) {
  const LP h = LP(0.5);
  LP gL = (Q.lap - P.lap) * inv_ds;
  LP gU = (Q.u - P.u) * inv_ds;
  LP c3 = h * (P.f0 + Q.f0) * inv_ds3 * sc;
  LP Bd = h * (P.f1 + Q.f1) * inv_ds * sc;
  LP wp = pl ? LP(1) : LP(0), wq = qr ? LP(1) : LP(0);
  dF[0] = -wp * c3;
  dF[1] = (LP(2) + wp) * c3 + h * sc * (P.d0 * gL + P.d1 * gU) - Bd;
  dF[2] = -(LP(2) + wq) * c3 + h * sc * (Q.d0 * gL + Q.d1 * gU) + Bd;
  dF[3] = wq * c3;
}

template <class LP> struct LUState {
  LP g1, d1, z1, g2, d2, z2;  // (gamma, delta, z) of rows i-1 and i-2
  __device__ __forceinline__ void reset() { g1 = d1 = z1 = g2 = d2 = z2 = LP(0); }
  // Eliminate row i (a x_{i-2} + b x_{i-1} + c x_i + d x_{i+1} + e x_{i+2} = r).
  // chk accumulates pivot * (1/pivot): it turns NaN, and stays NaN, once a
  // pivot is zero or non-finite, so callers test it once per chunk.
  __device__ __forceinline__ void step(LP a, LP b, LP c, LP d, LP e, LP r, LP& g, LP& dl, LP& z, LP& chk) {
    LP beta = b - a * g2;
    LP mu = c - a * d2 - beta * g1;
    LP inv = rcp(mu);
    g = (d - beta * d1) * inv;
    dl = e * inv;
    z = (r - a * z2 - beta * z1) * inv;
    g2 = g1;
    d2 = d1;
    z2 = z1;
    g1 = g;
    d1 = dl;
    z1 = z;
    chk = fma(mu, inv, chk);
  }
};

template <class LP>
__device__ __forceinline__ void band_row(const LP L[4], const LP R[4], LP& a, LP& b, LP& c, LP& d,
                                         LP& e) {
  a = -L[0];
  b = R[0] - L[1];
  c = LP(1) + R[1] - L[2];
  d = R[2] - L[3];
  e = R[3];
}

// ---------------------------------------------------------------------------
// per-cell helpers of the update and the Newton test

__device__ __forceinline__ double rel_update(double v, double uk) { return fabs(v / uk); }
__device__ __forceinline__ float rel_update(float v, double uk) {
  return __fdividef(fabsf(v), f32_of_pos_f64_fast(uk));  // uk > 0 or the step fails anyway
}
// Order-preserving integer key of a non-negative double (bit pattern);
// negative values, zero, NaN and infinities are reported separately.
__device__ __forceinline__ bool positive_finite_bits(double u) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(u);
  return (b >> 63) == 0 && b != 0ull && ((b >> 52) & 0x7ff) != 0x7ff;
}

// ---------------------------------------------------------------------------
// Reductions over the per-block partials (one block, fixed order).

// The reduction of the per-block partials into the iteration's scalars by
// one block of 256 threads: thread 0 writes *out and returns true.
__device__ __forceinline__ bool finalize_block(const PartX* __restrict__ px, int nx_part,
                                               const PartY* __restrict__ py, int ny_part,
                                               Scalars* __restrict__ out) {
  __shared__ double s_err[256], s_g[256], s_h[256];
  __shared__ Mass128 s_m[256];
  __shared__ int s_nf[256], s_pv[256];
  const int t = threadIdx.x;
  double err = 0.0, g = 0.0, h = INFINITY;
  Mass128 m = {0ull, 0ull};
  int nf = 0, pv = 0;
  for (int k = t; k < nx_part; k += 256) {
    if (!(px[k].gnorm <= g)) g = px[k].gnorm;
    pv |= px[k].pivot;
  }
  for (int k = t; k < ny_part; k += 256) {
    if (!(py[k].err <= err)) err = py[k].err;
    h = fmin(h, py[k].hmin);
    mass_add(m, py[k].mass);
    nf |= py[k].nonfinite;
    pv |= py[k].pivot;
  }
  s_err[t] = err;
  s_g[t] = g;
  s_h[t] = h;
  s_m[t] = m;
  s_nf[t] = nf;
  s_pv[t] = pv;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (t < o) {
      if (!(s_err[t + o] <= s_err[t])) s_err[t] = s_err[t + o];
      if (!(s_g[t + o] <= s_g[t])) s_g[t] = s_g[t + o];
      s_h[t] = fmin(s_h[t], s_h[t + o]);
      mass_add(s_m[t], s_m[t + o]);
      s_nf[t] |= s_nf[t + o];
      s_pv[t] |= s_pv[t + o];
    }
    __syncthreads();
  }
  if (t == 0) {
    Scalars s;
    s.err = s_err[0];
    s.gnorm = s_g[0];
    s.hmin = s_h[0];
    s.mass = s_m[0];
    s.nonfinite = s_nf[0];
    s.pivot = s_pv[0];
    *out = s;
    return true;
  }
  return false;
}

static __global__ void __launch_bounds__(256)
    k_finalize(const PartX* __restrict__ px, int nx_part, const PartY* __restrict__ py, int ny_part,
               Scalars* __restrict__ out) {
  finalize_block(px, nx_part, py, ny_part, out);
}

// Mass and minimum of a grid (for tf_residual's norms).
static __global__ void __launch_bounds__(256)
    k_grid_stats(const double* __restrict__ u, size_t N, PartY* __restrict__ part,
                 const double* const* __restrict__ up = nullptr) {
  if (up) u = *up;  // the grid named by a device-resident pointer (ensemble graphs)
  // min over positive values through their bit patterns (integer compares)
  unsigned long long hb = 0x7ff0000000000000ull;
  Mass128 m = {0ull, 0ull};
  int nf = 0;
  auto take = [&](double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    if (!positive_finite_bits(v)) nf = 1;
    else if (b < hb) hb = b;
    mass_add(m, (unsigned long long)fixed36_of_f64(v));
  };
  const size_t T = (size_t)gridDim.x * blockDim.x, t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  size_t done = 0;
  if ((reinterpret_cast<uintptr_t>(u) & 15) == 0) {
    // 16-byte loads, two per thread in flight: this pass is bound by the
    // HBM latency of its loads, not by their number
    const double2* u2 = reinterpret_cast<const double2*>(u);
    const size_t N4 = N / 4;
    for (size_t k = t0; k < N4; k += T) {
      const double2 a = __ldg(u2 + 2 * k), c = __ldg(u2 + 2 * k + 1);
      take(a.x);
      take(a.y);
      take(c.x);
      take(c.y);
    }
    done = 4 * N4;
  }
  for (size_t k = done + t0; k < N; k += T) take(__ldg(u + k));
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long h2 = __shfl_xor_sync(0xffffffffu, hb, o);
    if (h2 < hb) hb = h2;
    Mass128 m2;
    m2.lo = __shfl_xor_sync(0xffffffffu, m.lo, o);
    m2.hi = __shfl_xor_sync(0xffffffffu, m.hi, o);
    mass_add(m, m2);
    nf |= __shfl_xor_sync(0xffffffffu, nf, o);
  }
  __shared__ unsigned long long sh[8];
  __shared__ Mass128 sm[8];
  __shared__ int sn[8];
  if ((threadIdx.x & 31) == 0) {
    sh[threadIdx.x >> 5] = hb;
    sm[threadIdx.x >> 5] = m;
    sn[threadIdx.x >> 5] = nf;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long hbb = sh[0];
    Mass128 mb = sm[0];
    int nb = sn[0];
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
      if (sh[k] < hbb) hbb = sh[k];
      mass_add(mb, sm[k]);
      nb |= sn[k];
    }
    PartY p;
    p.err = 0.0;
    p.hmin = __longlong_as_double((long long)hbb);
    p.mass = mb;
    p.nonfinite = nb;
    p.pivot = 0;
    part[blockIdx.x] = p;
  }
}

template <class T>
__global__ void k_to_f64(const T* __restrict__ x, double* __restrict__ y, size_t N) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x)
    y[k] = to_f64(x[k]);
}

}  // namespace tf
