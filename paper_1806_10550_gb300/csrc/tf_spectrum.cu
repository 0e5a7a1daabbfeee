// tf_spectrum.cu -- radial Fourier analysis of a film on the GPU (App. Radial
// Fourier Transform): the dominant wavenumber of a film pattern.
//
// Steps (the appendix's order; the readings are those stated in tf.h):
//   1. A[q][p] = |C[q][p]| / (nx ny), C the 2-D DCT-II sum of zeta = h - H0,
//      i.e. the FFT magnitude of the film reflected evenly about its walls.
//      Each 1-D DCT-II of length n (a power of two) is Makhoul's reordering
//      v = (x0, x2, x4, ..., x5, x3, x1), one complex FFT of length n in
//      shared memory (Stockham passes of radix 16 in registers, then one of
//      radix 2, 4 or 8), and
//      the rotation C_k = Re(exp(-i pi k / 2n) V_k).  Two real lines ride in
//      one complex FFT (real and imaginary parts) and are separated with
//      V1 = (Z_k + conj Z_{n-k}) / 2, V2 = (Z_k - conj Z_{n-k}) / 2i.
//      Rows first (only the wave indices the later steps read are written),
//      then the columns of that narrow block.  FP32 arithmetic with
//      twiddles rounded from FP64; zeta is formed without FP64 arithmetic.
//   2. Gaussian smoothing along p, then along q (FP64), with the reflected
//      film's spectrum continued outside the index range.
//   3-4. Mean over each group of equal |q| (integer keys).  The grouping is
//      geometry only, so the plan builds it once: a counting sort of the
//      block's points by key, members of each group in ascending (q, p)
//      order, so that every run sums a group in the same order.
//   5-7. The least-squares normal equations of the continuous
//      piecewise-linear fit (tridiagonal, assembled per unknown without
//      atomics, solved by block elimination over many SMs plus parallel
//      cyclic reduction on the separators); then one block samples the fit
//      at n_eval points, smooths it and finds the roots of its derivative.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include "tf.h"

namespace {

constexpr int kFitThreads = 1024;
constexpr int kMaxLine = 16384;           // longest line a DCT handles
constexpr int kLineBuffer = 8192;         // complex values per FFT block at least
constexpr long long kMaxKeys = 1LL << 27; // largest key range of the radial grouping
constexpr int kMaxEval = 4096;           // largest n_eval

enum { kRows, kCols, kSmoothP, kSmoothQ, kRadial, kFit, kKernels };  // timed groups

inline bool pow2(int n) { return n >= 1 && (n & (n - 1)) == 0; }
inline int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

// ---- step 1: line DCTs -------------------------------------------------------
__device__ __forceinline__ int makhoul_slot(int i, int n) {
  return (i & 1) ? n - 1 - (i >> 1) : (i >> 1);
}

// zeta = h - H0 in FP32 without FP64 arithmetic or conversions (the FP64
// pipe is narrow): h = hi + lo, hi the float with h's sign, exponent and top
// 23 fraction bits (exact), lo the next 23 fraction bits (exact: the 2^23
// trick, 2^23 + m - 2^23, scaled by a power of two), the last 6 bits
// dropped (below 2^-46 |h|).  With H0 = H0hi + H0lo (H0hi = fl32(H0), the
// host rounds the rest), (hi - H0hi) + (lo - H0lo) is within
// 2^-24 |zeta| + 2^-45 (|h| + |H0|) of zeta.  Heights outside
// [2^-68, 2^128) take the FP64 route.
// The fast path alone; ok is false where h needs the FP64 route.
__device__ __forceinline__ float zeta_fast(double h, float H0hi, float H0lo, bool& ok) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(h);
  const unsigned hi32 = (unsigned)(bits >> 32), lo32 = (unsigned)bits;
  const int e = (int)((hi32 >> 20) & 0x7ffu);
  ok = e >= 955 && e <= 1150;
  const unsigned sign = hi32 & 0x80000000u;
  const float fh = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | ((hi32 & 0xfffffu) << 3) | (lo32 >> 29));
  // bits 28..6 of the fraction, worth m 2^(e-1069)
  const float m = __uint_as_float(0x4b000000u | ((lo32 >> 6) & 0x7fffffu)) - 8388608.0f;
  const float sc = __uint_as_float(sign | ((unsigned)(e - 942) << 23));
  return (fh - H0hi) + (m * sc - H0lo);
}

__device__ __forceinline__ float zeta_f32(double h, double H0, float H0hi, float H0lo) {
  bool ok;
  const float z = zeta_fast(h, H0hi, H0lo, ok);
  return ok ? z : (float)(h - H0);
}

// Shared-memory index with one pad slot per 16 values, so that the strided
// accesses of the early passes fall into different banks.
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// v * exp(-2 pi i k / 16) for k < 8; k is a constant once the callers'
// loops are unrolled, so the switch folds to the one case, with the
// products by 1, -i and sqrt(1/2) (1 - i) written out.
__device__ __forceinline__ float2 mul_w16(float2 v, int k) {
  const float C1 = 0.92387953251128674f;  // cos(pi/8)
  const float S1 = 0.38268343236508977f;  // sin(pi/8)
  const float R2 = 0.70710678118654752f;  // sqrt(1/2)
  switch (k) {
    case 0: return v;
    case 1: return make_float2(C1 * v.x + S1 * v.y, C1 * v.y - S1 * v.x);
    case 2: return make_float2(R2 * (v.x + v.y), R2 * (v.y - v.x));
    case 3: return make_float2(S1 * v.x + C1 * v.y, S1 * v.y - C1 * v.x);
    case 4: return make_float2(v.y, -v.x);
    case 5: return make_float2(C1 * v.y - S1 * v.x, -S1 * v.y - C1 * v.x);
    case 6: return make_float2(R2 * (v.y - v.x), -R2 * (v.x + v.y));
    default: return make_float2(S1 * v.y - C1 * v.x, -C1 * v.y - S1 * v.x);
  }
}

// In-register forward DFT of length R (2, 4, 8 or 16): radix-2 decimation
// in time on a compile-time permuted array, output in natural order.
template <int R>
__device__ __forceinline__ void dft_regs(float2 (&v)[R]) {
  constexpr int L = R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4;
  float2 x[R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    int r = 0;
#pragma unroll
    for (int b = 0; b < L; ++b) r |= ((i >> b) & 1) << (L - 1 - b);
    x[r] = v[i];
  }
#pragma unroll
  for (int m = 1; m < R; m <<= 1) {
#pragma unroll
    for (int i = 0; i < R; ++i) {
      if ((i & m) == 0) {
        const int pos = i & (m - 1);
        const float2 t = mul_w16(x[i + m], pos * (8 / m));  // times exp(-2 pi i pos / 2m)
        x[i + m] = make_float2(x[i].x - t.x, x[i].y - t.y);
        x[i] = make_float2(x[i].x + t.x, x[i].y + t.y);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < R; ++i) v[i] = x[i];
}

// One Stockham pass of radix R over G lines of length n = 2^lg stored back to
// back (padded): p is the length of the sub-transforms already formed.
// Sub-transform column j (k = j mod p) takes x[j + r n/R], twiddles it by
// exp(-2 pi i r k / pR) and writes its R-point DFT to (j - k) R + k + s p.
// Every thread handles 16/R columns; reads finish before writes (in place).
template <int R, int THREADS>
__device__ __forceinline__ void stockham_pass(float2* buf, int n, int lg, int p,
                                              const float2* __restrict__ tw) {
  constexpr int JPT = 16 / R;
  constexpr int LR = R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4;
  const int cols = n >> LR, lgc = lg - LR;
  float2 v[JPT][R];
  int out_base[JPT];
#pragma unroll
  for (int jj = 0; jj < JPT; ++jj) {
    const int jg = threadIdx.x + jj * THREADS;
    const int g = jg >> lgc, j = jg & (cols - 1), k = j & (p - 1);
    const int base = g << lg;
#pragma unroll
    for (int r = 0; r < R; ++r) v[jj][r] = buf[pad16(base + j + r * cols)];
    if (p > 1) {  // twiddles exp(-2 pi i r k / pR) = tw[r k n / pR]: powers
                  // 1, 2, 4, 8 from the table, the others as their products
      const int step = k * (n / (p * R));
      const float2 w1 = __ldg(&tw[step]);
      v[jj][1] = cmul(v[jj][1], w1);
      if (R > 2) {
        const float2 w2 = __ldg(&tw[2 * step]);
        v[jj][2] = cmul(v[jj][2], w2);
        v[jj][3] = cmul(v[jj][3], cmul(w1, w2));
        if (R > 4) {
          const float2 w4 = __ldg(&tw[4 * step]);
#pragma unroll
          for (int r = 4; r < 8; ++r) {
            float2 w = w4;
            if (r & 1) w = cmul(w, w1);
            if (r & 2) w = cmul(w, w2);
            v[jj][r] = cmul(v[jj][r], w);
          }
          if (R > 8) {
            const float2 w8 = __ldg(&tw[8 * step]);
#pragma unroll
            for (int r = 8; r < 16; ++r) {
              float2 w = w8;
              if (r & 1) w = cmul(w, w1);
              if (r & 2) w = cmul(w, w2);
              if (r & 4) w = cmul(w, w4);
              v[jj][r] = cmul(v[jj][r], w);
            }
          }
        }
      }
    }
    dft_regs<R>(v[jj]);
    out_base[jj] = base + (j - k) * R + k;
  }
  __syncthreads();
#pragma unroll
  for (int jj = 0; jj < JPT; ++jj) {
#pragma unroll
    for (int s = 0; s < R; ++s) buf[pad16(out_base[jj] + s * p)] = v[jj][s];
  }
  __syncthreads();
}

// Forward FFT of every length-n line in buf (16 * THREADS values in all),
// natural order in and out.  tw[k] = exp(-2 pi i k / n), k < n.
// The passes start after the first l0 bits (sub-transforms of length 2^l0
// already formed).
template <int THREADS>
__device__ __forceinline__ void fft_lines(float2* buf, int n, int lg, const float2* __restrict__ tw, int l0 = 0) {
  int p = 1 << l0, l = l0;
  for (; l + 4 <= lg; l += 4, p <<= 4) stockham_pass<16, THREADS>(buf, n, lg, p, tw);
  switch (lg - l) {
    case 1: stockham_pass<2, THREADS>(buf, n, lg, p, tw); break;
    case 2: stockham_pass<4, THREADS>(buf, n, lg, p, tw); break;
    case 3: stockham_pass<8, THREADS>(buf, n, lg, p, tw); break;
    default: break;
  }
}

// The two real DCT-II outputs at index k of the line pair held in z
// (padded indices, line base zb).
__device__ __forceinline__ void dct_pair(const float2* buf, int zb, int n, int k, float2 rot, float& c1,
                                         float& c2) {
  const float2 Z = buf[pad16(zb + k)], Zc = buf[pad16(zb + ((n - k) & (n - 1)))];
  const float v1x = 0.5f * (Z.x + Zc.x), v1y = 0.5f * (Z.y - Zc.y);
  const float v2x = 0.5f * (Z.y + Zc.y), v2y = -0.5f * (Z.x - Zc.x);
  c1 = rot.x * v1x - rot.y * v1y;
  c2 = rot.x * v2x - rot.y * v2y;
}

// Rows: h [ny][nx] (FP64) -> X [ny][Pb] (FP32), X[r][k] = sum_i zeta[r][i]
// cos(pi k (2i+1) / 2nx) for k < Pb.  Block b handles the G = 16 THREADS / nx
// row pairs b*G .. b*G+G-1 (rows 2 pair, 2 pair + 1).
template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) k_dct_rows(const double* __restrict__ h, int nx, int ny,
                                                      double H0, float H0hi, float H0lo, int lg, int Pb,
                                                      const float2* __restrict__ tw,
                                                      const float2* __restrict__ rot,
                                                      float* __restrict__ X) {
  extern __shared__ float2 zbuf[];
  const int G = (16 * THREADS) >> lg;
  const int pair0 = blockIdx.x * G;
  int l0 = 0;
  if (nx >= 4 && (reinterpret_cast<uintptr_t>(h) & 15) == 0) {
    // Makhoul order v[j] = x[2j], v[n-1-j] = x[2j+1].  The value pairs at 2j
    // and n-2-2j (j < n/4) give v[j], v[n-1-j], v[n/2-1-j] and v[n/2+j]:
    // both inputs of the first radix-2 pass for columns j and n/2-1-j, done
    // here in registers (Stockham, p = 1: outputs 2c and 2c+1 of column c).
    const double2* h2 = reinterpret_cast<const double2*>(h);
    const int half = nx >> 1, quarter = nx >> 2;
#pragma unroll 1
    for (int q0 = 0; q0 < 4; q0 += 2) {
      double2 a0[2], b0[2], a1[2], b1[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int e4 = threadIdx.x + (q0 + q) * THREADS;
        const int g = e4 >> (lg - 2), j = e4 & (quarter - 1);
        const int r0 = 2 * (pair0 + g), r1 = r0 + 1;
        const double2 fill = make_double2(H0, H0);
        a0[q] = r0 < ny ? h2[(size_t)r0 * half + j] : fill;
        b0[q] = r0 < ny ? h2[(size_t)r0 * half + half - 1 - j] : fill;
        a1[q] = r1 < ny ? h2[(size_t)r1 * half + j] : fill;
        b1[q] = r1 < ny ? h2[(size_t)r1 * half + half - 1 - j] : fill;
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int e4 = threadIdx.x + (q0 + q) * THREADS;
        const int g = e4 >> (lg - 2), j = e4 & (quarter - 1);
        const int base = g << lg, jc = half - 1 - j;
        // (row r0 real, row r1 imaginary); the FP64 route only when a lane
        // of the warp needs it (a uniform branch, not run otherwise)
        bool ok[8];
        float2 vj = make_float2(zeta_fast(a0[q].x, H0hi, H0lo, ok[0]), zeta_fast(a1[q].x, H0hi, H0lo, ok[1]));
        float2 vn = make_float2(zeta_fast(a0[q].y, H0hi, H0lo, ok[2]), zeta_fast(a1[q].y, H0hi, H0lo, ok[3]));
        float2 vc = make_float2(zeta_fast(b0[q].x, H0hi, H0lo, ok[4]), zeta_fast(b1[q].x, H0hi, H0lo, ok[5]));
        float2 vh = make_float2(zeta_fast(b0[q].y, H0hi, H0lo, ok[6]), zeta_fast(b1[q].y, H0hi, H0lo, ok[7]));
        const bool all_ok = ok[0] && ok[1] && ok[2] && ok[3] && ok[4] && ok[5] && ok[6] && ok[7];
        if (__any_sync(0xffffffffu, !all_ok)) {
          vj = make_float2(zeta_f32(a0[q].x, H0, H0hi, H0lo), zeta_f32(a1[q].x, H0, H0hi, H0lo));
          vn = make_float2(zeta_f32(a0[q].y, H0, H0hi, H0lo), zeta_f32(a1[q].y, H0, H0hi, H0lo));
          vc = make_float2(zeta_f32(b0[q].x, H0, H0hi, H0lo), zeta_f32(b1[q].x, H0, H0hi, H0lo));
          vh = make_float2(zeta_f32(b0[q].y, H0, H0hi, H0lo), zeta_f32(b1[q].y, H0, H0hi, H0lo));
        }
        // column j: v[j] +- v[j + n/2] (= vh); column jc: v[jc] (= vc) +- v[jc + n/2] (= vn)
        zbuf[pad16(base + 2 * j)] = make_float2(vj.x + vh.x, vj.y + vh.y);
        zbuf[pad16(base + 2 * j + 1)] = make_float2(vj.x - vh.x, vj.y - vh.y);
        zbuf[pad16(base + 2 * jc)] = make_float2(vc.x + vn.x, vc.y + vn.y);
        zbuf[pad16(base + 2 * jc + 1)] = make_float2(vc.x - vn.x, vc.y - vn.y);
      }
    }
    l0 = 1;
  } else {
    for (int e = threadIdx.x; e < G * nx; e += THREADS) {
      const int g = e >> lg, i = e & (nx - 1);
      const int r0 = 2 * (pair0 + g), r1 = r0 + 1;
      float a = 0.f, b = 0.f;
      if (r0 < ny) a = zeta_f32(h[(size_t)r0 * nx + i], H0, H0hi, H0lo);
      if (r1 < ny) b = zeta_f32(h[(size_t)r1 * nx + i], H0, H0hi, H0lo);
      zbuf[pad16((g << lg) + makhoul_slot(i, nx))] = make_float2(a, b);
    }
  }
  __syncthreads();
  fft_lines<THREADS>(zbuf, nx, lg, tw, l0);
  for (int e = threadIdx.x; e < G * Pb; e += THREADS) {
    const int g = e / Pb, k = e - g * Pb;
    const int r0 = 2 * (pair0 + g), r1 = r0 + 1;
    float c1, c2;
    dct_pair(zbuf, g << lg, nx, k, __ldg(&rot[k]), c1, c2);
    if (r0 < ny) X[(size_t)r0 * Pb + k] = c1;
    if (r1 < ny) X[(size_t)r1 * Pb + k] = c2;
  }
}

// Columns: X [ny][Pb] -> A [Qb][Pb] (FP64), A = |C| * inv.  Block b handles
// the G = 16 THREADS / ny column pairs b*G .. b*G+G-1 (columns 2 pair,
// 2 pair + 1).
template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) k_dct_cols(const float* __restrict__ X, int ny, int Pb, int Qb,
                                                      int lg, const float2* __restrict__ tw,
                                                      const float2* __restrict__ rot, double inv,
                                                      double* __restrict__ A) {
  extern __shared__ float2 zbuf[];
  const int G = (16 * THREADS) >> lg;
  const int c00 = 2 * blockIdx.x * G, W = 2 * G;
  // consecutive threads read consecutive columns of one row; W ny = 32
  // THREADS values, eight per thread in flight
#pragma unroll 1
  for (int q0 = 0; q0 < 32; q0 += 8) {
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = threadIdx.x + (q0 + q) * THREADS;
      const int i = e / W, c = c00 + (e - i * W);
      v[q] = c < Pb ? X[(size_t)i * Pb + c] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = threadIdx.x + (q0 + q) * THREADS;
      const int i = e / W, cl = e - i * W;
      float* slot = reinterpret_cast<float*>(&zbuf[pad16(((cl >> 1) << lg) + makhoul_slot(i, ny))]);
      slot[cl & 1] = v[q];
    }
  }
  __syncthreads();
  fft_lines<THREADS>(zbuf, ny, lg, tw);
  for (int e = threadIdx.x; e < G * Qb; e += THREADS) {
    const int k = e / G, g = e - k * G;
    const int c0 = c00 + 2 * g, c1i = c0 + 1;
    float c1, c2;
    dct_pair(zbuf, g << lg, ny, k, __ldg(&rot[k]), c1, c2);
    if (c0 < Pb) A[(size_t)k * Pb + c0] = fabs((double)c1) * inv;
    if (c1i < Pb) A[(size_t)k * Pb + c1i] = fabs((double)c2) * inv;
  }
}

// ---- step 2: Gaussian smoothing --------------------------------------------
// Index k of the reflected film's spectrum (period 2n): the stored index, or
// -1 where the spectrum is zero (k = n modulo 2n).
__device__ __forceinline__ int fold_index(int k, int n) {
  int m = k % (2 * n);
  if (m < 0) m += 2 * n;
  if (m < n) return m;
  if (m == n) return -1;
  return 2 * n - m;
}

// T[q][p] = sum_d w[d] A[q][fold(p + d)], q < Qb, p < n_p.
__global__ void k_smooth_p(const double* __restrict__ A, int Pb, int Qb, int n_p, int nx, int R,
                           const double* __restrict__ w, double* __restrict__ T) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y;
  if (p >= n_p || q >= Qb) return;
  double acc = 0.0;
  for (int d = -R; d <= R; ++d) {
    const int k = fold_index(p + d, nx);
    if (k >= 0) acc += w[d + R] * A[(size_t)q * Pb + k];
  }
  T[(size_t)q * n_p + p] = acc;
}

// S[q][p] = sum_d w[d] T[fold(q + d)][p], q < n_q, p < n_p.
__global__ void k_smooth_q(const double* __restrict__ T, int n_p, int n_q, int ny, int R,
                           const double* __restrict__ w, double* __restrict__ S) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y;
  if (p >= n_p || q >= n_q) return;
  double acc = 0.0;
  for (int d = -R; d <= R; ++d) {
    const int k = fold_index(q + d, ny);
    if (k >= 0) acc += w[d + R] * T[(size_t)k * n_p + p];
  }
  S[(size_t)q * n_p + p] = acc;
}

// ---- steps 3-4: radial grouping (plan) and means (run) ---------------------
__device__ __forceinline__ long long radial_key(int p, int q, int ax, int ay) {
  const long long a = (long long)p * ax, b = (long long)q * ay;
  return a * a + b * b;
}

__global__ void k_keys_count(int n_p, int n_q, int ax, int ay, long long keycut, int* __restrict__ cnt) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y;
  if (p >= n_p || q >= n_q) return;
  const long long k = radial_key(p, q, ax, ay);
  if (k <= keycut) atomicAdd(&cnt[k], 1);
}

// One block: koff[key] = points with smaller keys; for the M non-empty keys
// in ascending order rkey[r] = key, roff[r] = koff[key]; roff[M] = points;
// meta[0] = M, meta[1] = points.
__global__ void __launch_bounds__(kFitThreads) k_keys_scan(const int* __restrict__ cnt, long long nkeys,
                                                           int* __restrict__ koff,
                                                           long long* __restrict__ rkey,
                                                           int* __restrict__ roff, int* __restrict__ meta) {
  __shared__ int s_pts[kFitThreads], s_ne[kFitThreads];
  const int t = threadIdx.x;
  const long long chunk = (nkeys + kFitThreads - 1) / kFitThreads;
  const long long lo = min(nkeys, (long long)t * chunk), hi = min(nkeys, lo + chunk);
  int pts = 0, ne = 0;
  for (long long k = lo; k < hi; ++k) {
    const int c = cnt[k];
    pts += c;
    ne += c > 0;
  }
  s_pts[t] = pts;
  s_ne[t] = ne;
  __syncthreads();
  // inclusive scans (Hillis-Steele)
  for (int d = 1; d < kFitThreads; d <<= 1) {
    const int a = t >= d ? s_pts[t - d] : 0, b = t >= d ? s_ne[t - d] : 0;
    __syncthreads();
    s_pts[t] += a;
    s_ne[t] += b;
    __syncthreads();
  }
  int off = s_pts[t] - pts, rank = s_ne[t] - ne;
  for (long long k = lo; k < hi; ++k) {
    const int c = cnt[k];
    koff[k] = off;
    if (c > 0) {
      rkey[rank] = k;
      roff[rank] = off;
      ++rank;
    }
    off += c;
  }
  if (t == kFitThreads - 1) {
    meta[0] = s_ne[t];
    meta[1] = s_pts[t];
    roff[s_ne[t]] = s_pts[t];
  }
}

__global__ void k_keys_fill(int n_p, int n_q, int ax, int ay, long long keycut, const int* __restrict__ koff,
                            int* __restrict__ fill, int* __restrict__ member) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y;
  if (p >= n_p || q >= n_q) return;
  const long long k = radial_key(p, q, ax, ay);
  if (k <= keycut) member[koff[k] + atomicAdd(&fill[k], 1)] = q * n_p + p;
}

// Members of each group in ascending (q, p) order; |q| of each group.
__global__ void k_keys_order(int M, const long long* __restrict__ rkey, const int* __restrict__ roff,
                             int* __restrict__ member, double scale, double* __restrict__ rq) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= M) return;
  const int a = roff[r], b = roff[r + 1];
  for (int i = a + 1; i < b; ++i) {
    const int v = member[i];
    int j = i - 1;
    while (j >= a && member[j] > v) {
      member[j + 1] = member[j];
      --j;
    }
    member[j + 1] = v;
  }
  rq[r] = scale * sqrt((double)rkey[r]);
}

__global__ void k_radial_mean(int M, const int* __restrict__ roff, const int* __restrict__ member,
                              const double* __restrict__ S, double* __restrict__ rv) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= M) return;
  const int a = roff[r], b = roff[r + 1];
  double acc = 0.0;
  for (int i = a; i < b; ++i) acc += S[member[i]];
  rv[r] = acc / (double)(b - a);
}

// ---- steps 5-7: fit, sampling, smoothing, maxima (one block) -----------------
struct FitArgs {
  int M, K, ppi, n_eval;
  double q_cut;
  const double* rq;
  const double* rv;
  double *t, *diag, *off, *rhs, *a;  // K + 1 each
  double *cp, *zz, *za, *zb;         // K + 1 each (block elimination)
  double *w0, *w1, *d, *s;           // n_eval each (curve stages)
  double *cq, *cv;                   // n_eval: samples and smoothed curve
  double *pq, *pv;                   // n_eval: maxima
  int* n_peaks;
};

__device__ __forceinline__ int interval_end(int j, int K, int M, int ppi) {
  return j == K - 1 ? M : (j + 1) * ppi;
}

// 1/k for the moving-average windows (k = 1..7).
__constant__ double c_inv_count[8] = {0.0, 1.0, 1.0 / 2, 1.0 / 3, 1.0 / 4, 1.0 / 5, 1.0 / 6, 1.0 / 7};

// Second-order difference of y at e (central inside, one-sided at the
// ends); i2dq = 1 / (2 dq).
__device__ __forceinline__ double diff2(const double* y, int e, int n, double i2dq) {
  if (e == 0) return (-3.0 * y[0] + 4.0 * y[1] - y[2]) * i2dq;
  if (e == n - 1) return (3.0 * y[n - 1] - 4.0 * y[n - 2] + y[n - 3]) * i2dq;
  return (y[e + 1] - y[e - 1]) * i2dq;
}

// Nodes and normal equations of the hat-function basis, one thread per
// unknown u = 1..K: t[u], diag[u], off[u] (coupling of u and u + 1; off[0]
// and off[K] are 0), rhs[u].
__global__ void k_fit_assemble(FitArgs f) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int K = f.K, M = f.M, ppi = f.ppi;
  if (u > K) return;
  auto node = [&](int j) { return j == 0 ? 0.0 : (j == K ? f.q_cut : f.rq[j * ppi]); };
  if (u == 1) {
    f.t[0] = 0.0;
    f.off[0] = 0.0;
  }
  f.t[u] = node(u);
  double d = 0.0, r = 0.0, o = 0.0;
  {  // interval u-1: the hat of node u rises, weight s
    const int j = u - 1;
    const double t0 = node(j), ih = 1.0 / (node(j + 1) - t0);
    for (int i = j * ppi; i < interval_end(j, K, M, ppi); ++i) {
      const double s = (f.rq[i] - t0) * ih;
      d += s * s;
      r += s * f.rv[i];
    }
  }
  if (u < K) {  // interval u: the hat of node u falls, weight 1 - s
    const int j = u;
    const double t0 = node(j), ih = 1.0 / (node(j + 1) - t0);
    for (int i = j * ppi; i < interval_end(j, K, M, ppi); ++i) {
      const double s = (f.rq[i] - t0) * ih;
      d += (1.0 - s) * (1.0 - s);
      r += (1.0 - s) * f.rv[i];
      o += (1.0 - s) * s;
    }
  }
  f.diag[u] = d;
  f.rhs[u] = r;
  f.off[u] = o;
}

// Partitioned solve of the symmetric positive definite tridiagonal system
// (FP64, spread over many SMs: the FP64 pipe is narrow).  Separators every
// c-th unknown (s_b = b c, b = 1..S, S < kReduced) split the unknowns into
// interior blocks (b c, (b+1) c).  Each block is eliminated by one thread
// for three right sides (rhs and its couplings to the left and right
// separators); that leaves a tridiagonal Schur complement on the
// separators, solved by parallel cyclic reduction in one block; every
// interior unknown is then recovered from its two separators.
constexpr int kReduced = 512;

__host__ __device__ __forceinline__ int fit_chunk(int K) { return max(2, (K + 1 + kReduced - 1) / kReduced); }

__global__ void k_fit_blocks(FitArgs f) {
  const int K = f.K, c = fit_chunk(K), S = K / c;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int first = b * c + 1, last = min((b + 1) * c - 1, K);
  if (b > S || first > last) return;
  const double* __restrict__ dg = f.diag;
  const double* __restrict__ of = f.off;
  const double* __restrict__ rh = f.rhs;
  double* __restrict__ cp = f.cp;
  double* __restrict__ zz = f.zz;
  double* __restrict__ za = f.za;
  double* __restrict__ zb = f.zb;
  // forward sweep, the next row's inputs loaded one row ahead
  double cpv = 0.0, zv = 0.0, av = 0.0, bv = 0.0, sub = 0.0;
  double dn = dg[first], rn = rh[first], on = first < last ? of[first] : 0.0;
  for (int u = first; u <= last; ++u) {
    const double d = dn, r = rn, o = on;
    if (u < last) {
      dn = dg[u + 1];
      rn = rh[u + 1];
      on = u + 1 < last ? of[u + 1] : 0.0;
    }
    const double inv = 1.0 / (d - sub * cpv);
    cpv = o * inv;
    zv = (r - sub * zv) * inv;
    av = ((u == first ? of[first - 1] : 0.0) - sub * av) * inv;
    bv = ((u == last ? of[last] : 0.0) - sub * bv) * inv;
    cp[u] = cpv;
    zz[u] = zv;
    za[u] = av;
    zb[u] = bv;
    sub = o;  // the next row's sub-diagonal is this row's coupling
  }
  // back substitution, the row below carried in registers
  double zn = zz[last], an = za[last], bnx = zb[last];
  for (int u = last - 1; u >= first; --u) {
    const double cu = cp[u];
    zn = zz[u] - cu * zn;
    an = za[u] - cu * an;
    bnx = zb[u] - cu * bnx;
    zz[u] = zn;
    za[u] = an;
    zb[u] = bnx;
  }
}

__global__ void __launch_bounds__(kReduced) k_fit_reduced(FitArgs f) {
  __shared__ double sl[kReduced], sd[kReduced], su[kReduced], sr[kReduced], si[kReduced];
  const int K = f.K, c = fit_chunk(K), S = K / c;
  const int b = threadIdx.x + 1;  // separator b (row b - 1 of the reduced system)
  if (threadIdx.x == 0) f.a[0] = 0.0;
  if (b <= S) {
    const int sp = b * c, pl = sp - 1, pr = sp + 1;
    const double eL = f.off[pl], eR = f.off[sp];
    double d = f.diag[sp] - eL * f.zb[pl];
    double r = f.rhs[sp] - eL * f.zz[pl];
    const double lw = b > 1 ? -eL * f.za[pl] : 0.0;
    double up = 0.0;
    if (pr <= K) {
      d -= eR * f.za[pr];
      r -= eR * f.zz[pr];
      up = b < S ? -eR * f.zb[pr] : 0.0;
    }
    sl[b - 1] = lw;
    sd[b - 1] = d;
    su[b - 1] = up;
    sr[b - 1] = r;
  }
  __syncthreads();
  const int i = threadIdx.x;
  for (int st = 1; st < S; st <<= 1) {
    if (i < S) si[i] = 1.0 / sd[i];
    __syncthreads();
    double nl = 0.0, nd = 0.0, nu = 0.0, nr = 0.0;
    if (i < S) {
      nd = sd[i];
      nr = sr[i];
      if (i - st >= 0) {
        const double al = -sl[i] * si[i - st];
        nd += al * su[i - st];
        nr += al * sr[i - st];
        nl = al * sl[i - st];
      }
      if (i + st < S) {
        const double ga = -su[i] * si[i + st];
        nd += ga * sl[i + st];
        nr += ga * sr[i + st];
        nu = ga * su[i + st];
      }
    }
    __syncthreads();
    if (i < S) {
      sl[i] = nl;
      sd[i] = nd;
      su[i] = nu;
      sr[i] = nr;
    }
    __syncthreads();
  }
  if (b <= S) f.a[b * c] = sr[b - 1] / sd[b - 1];
}

__global__ void k_fit_back(FitArgs f) {
  const int K = f.K, c = fit_chunk(K);
  const int u = blockIdx.x * blockDim.x + threadIdx.x + 1;
  if (u > K || u % c == 0) return;
  const int b = u / c;
  const double xL = b >= 1 ? f.a[b * c] : 0.0;
  const double xR = (b + 1) * c <= K ? f.a[(b + 1) * c] : 0.0;
  f.a[u] = f.zz[u] - f.za[u] * xL - f.zb[u] * xR;
}

// One block: sampling, moving averages, derivatives and maxima.  Global
// memory written by the block is read back after __syncthreads, which makes
// it visible within the block.
__global__ void __launch_bounds__(kFitThreads) k_fit_peaks(FitArgs f) {
  const int K = f.K, n = f.n_eval;
  // the fitted curve at n equispaced points of [0, q_cut]
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const double q = f.q_cut * (double)e / (double)(n - 1);
    double y;
    if (q >= f.t[K]) {
      y = f.a[K];
    } else {
      int lo = 0, hi = K;  // t[lo] <= q < t[hi]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (f.t[mid] <= q) lo = mid;
        else hi = mid;
      }
      const double slope = (f.a[lo + 1] - f.a[lo]) / (f.t[lo + 1] - f.t[lo]);
      y = slope * (q - f.t[lo]) + f.a[lo];
    }
    f.cq[e] = q;
    f.w0[e] = y;
  }
  __syncthreads();
  // moving averages of half-widths 3, 2, 1 (windows cut at the ends)
  double* src = f.w0;
  double* dst = f.w1;
  for (int P = 3; P >= 1; --P) {
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int lo = max(0, e - P), hi = min(n - 1, e + P);
      double acc = 0.0;
      for (int i = lo; i <= hi; ++i) acc += src[i];
      dst[e] = acc * c_inv_count[hi - lo + 1];
    }
    __syncthreads();
    double* tmp = src;
    src = dst;
    dst = tmp;
  }
  const double i2dq = (double)(n - 1) / (2.0 * f.q_cut);
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    f.cv[e] = src[e];
    f.d[e] = diff2(src, e, n, i2dq);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n; e += blockDim.x) f.s[e] = diff2(f.d, e, n, i2dq);
  __syncthreads();
  // maxima: candidates in any order (w0, w1), then each placed by its rank
  // (highest value first, ties by wavenumber)
  __shared__ int s_np;
  if (threadIdx.x == 0) s_np = 0;
  __syncthreads();
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const double* d = f.d;
    double fr;
    if (d[e] == 0.0) fr = 0.0;
    else if (e + 1 < n && ((d[e] > 0.0 && d[e + 1] < 0.0) || (d[e] < 0.0 && d[e + 1] > 0.0)))
      fr = d[e] / (d[e] - d[e + 1]);
    else continue;
    const int e1 = min(e + 1, n - 1);
    const double sr = f.s[e] + fr * (f.s[e1] - f.s[e]);
    if (sr < 0.0) {
      const int slot = atomicAdd(&s_np, 1);
      f.w0[slot] = f.cq[e] + fr * (f.cq[e1] - f.cq[e]);
      f.w1[slot] = f.cv[e] + fr * (f.cv[e1] - f.cv[e]);
    }
  }
  __syncthreads();
  const int np = s_np;
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    const double qi = f.w0[i], vi = f.w1[i];
    int rank = 0;
    for (int j = 0; j < np; ++j) rank += (f.w1[j] > vi) || (f.w1[j] == vi && f.w0[j] < qi);
    f.pq[rank] = qi;
    f.pv[rank] = vi;
  }
  if (threadIdx.x == 0) *f.n_peaks = np;
}

// ---- host side ---------------------------------------------------------------
template <typename T>
T* carve(unsigned char*& cur, size_t count) {
  T* p = reinterpret_cast<T*>(cur);
  cur += ((count * sizeof(T) + 255) / 256) * 256;
  return p;
}

// Dynamic shared memory of an FFT block of THREADS threads (16 values each, padded).
size_t fft_smem(int threads) { return sizeof(float2) * (size_t)(16 * threads + threads); }

long long isqrt_ll(long long v) {
  long long r = (long long)floor(sqrt((double)v));
  while (r > 0 && r * r > v) --r;
  while ((r + 1) * (r + 1) <= v) ++r;
  return r;
}

long long gcd_ll(long long a, long long b) {
  while (b) {
    const long long t = a % b;
    a = b;
    b = t;
  }
  return a;
}

// tw[k] = exp(-2 pi i k / n), rot[k] = exp(-i pi k / 2n), k < n.
void host_tables(int n, float2* tw, float2* rot) {
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < n; ++k) {
    const double a = -2.0 * pi * (double)k / (double)n;
    tw[k] = make_float2((float)cos(a), (float)sin(a));
  }
  for (int k = 0; k < n; ++k) {
    const double a = -pi * (double)k / (2.0 * (double)n);
    rot[k] = make_float2((float)cos(a), (float)sin(a));
  }
}

}  // namespace

struct tf_spectrum_plan {
  int nx, ny, lgx, lgy, thx, thy;
  double ds;
  tf_spectrum_params sp;
  cudaStream_t stream;
  int R, n_p, n_q, Pb, Qb, M, K, npts;
  int ax, ay;
  long long keycut;
  double scale;
  unsigned char* arena;
  float2 *twx, *rotx, *twy, *roty;
  double* w;
  float* X;
  double *A, *T, *S;
  int *member, *roff;
  double *rq, *rv;
  double *t, *diag, *off, *rhs, *a, *cp, *zz, *za, *zb;
  double *w0, *w1, *dd, *ss, *cq, *cv, *pq, *pv;
  int* d_npeaks;
  cudaEvent_t ev[kKernels + 1];
  float ms[kKernels];
};

extern "C" {

void tf_spectrum_params_default(tf_spectrum_params* sp) {
  if (!sp) return;
  memset(sp, 0, sizeof(*sp));
  sp->H0 = 1.0;
  sp->q_cut = 0.0;
  sp->sigma = 1.0;
  sp->points_per_interval = 10;
  sp->n_eval = 400;
}

void tf_spectrum_plan_destroy(tf_spectrum_plan* P) {
  if (!P) return;
  for (int i = 0; i <= kKernels; ++i)
    if (P->ev[i]) cudaEventDestroy(P->ev[i]);
  if (P->arena) cudaFree(P->arena);
  free(P);
}

int tf_spectrum_plan_create(int nx, int ny, double ds, const tf_spectrum_params* sp, void* stream,
                            tf_spectrum_plan** out) {
  if (!out) return TF_ERR_ARG;
  *out = nullptr;
  if (!sp || !pow2(nx) || !pow2(ny) || nx > kMaxLine || ny > kMaxLine) return TF_ERR_ARG;
  if (!(ds > 0.0) || !isfinite(ds) || !(sp->q_cut > 0.0) || !isfinite(sp->q_cut)) return TF_ERR_ARG;
  if (!(sp->sigma >= 0.0) || sp->sigma > 16.0 || sp->points_per_interval < 1) return TF_ERR_ARG;
  if (sp->n_eval < 3 || sp->n_eval > kMaxEval || !isfinite(sp->H0)) return TF_ERR_ARG;

  tf_spectrum_plan* P = (tf_spectrum_plan*)calloc(1, sizeof(tf_spectrum_plan));
  if (!P) return TF_ERR_NOMEM;
  P->nx = nx;
  P->ny = ny;
  P->ds = ds;
  P->sp = *sp;
  P->stream = (cudaStream_t)stream;
  P->lgx = ilog2(nx);
  P->lgy = ilog2(ny);
  P->thx = std::max(nx, kLineBuffer) / 16;  // FFT block: 16 values per thread
  P->thy = std::max(ny, kLineBuffer) / 16;
  P->R = sp->sigma > 0.0 ? (int)ceil(3.0 * sp->sigma) : 0;
  // radial geometry: key = (p ax)^2 + (q ay)^2, |q| = scale sqrt(key)
  const long long g = gcd_ll(nx, ny);
  P->ax = (int)(ny / g);
  P->ay = (int)(nx / g);
  P->scale = 3.14159265358979323846 * (double)g / (ds * nx * ny);
  const double r = sp->q_cut / P->scale;
  const double kc = floor(r * r);
  if (!(kc < (double)kMaxKeys)) {
    free(P);
    return TF_ERR_ARG;
  }
  P->keycut = (long long)kc;
  const long long root = isqrt_ll(P->keycut);
  P->n_p = (int)std::min<long long>(nx, root / P->ax + 1);
  P->n_q = (int)std::min<long long>(ny, root / P->ay + 1);
  P->Pb = std::min(nx, P->n_p + P->R);
  P->Qb = std::min(ny, P->n_q + P->R);
  const long long nkeys = P->keycut + 1;
  const size_t blk = (size_t)P->n_p * P->n_q;
  const size_t max_groups = (size_t)std::min<long long>(nkeys, (long long)blk);
  const int n = sp->n_eval;

  // workspace (fit arrays sized by the largest possible group count)
  const size_t max_K = max_groups + 1;
  size_t bytes = 0;
  auto add = [&](size_t cnt, size_t sz) { bytes += ((cnt * sz + 255) / 256) * 256; };
  add(nx, sizeof(float2));
  add(nx, sizeof(float2));
  add(ny, sizeof(float2));
  add(ny, sizeof(float2));
  add(2 * P->R + 1, sizeof(double));
  add((size_t)ny * P->Pb, sizeof(float));
  add((size_t)P->Qb * P->Pb, sizeof(double));
  add((size_t)P->Qb * P->n_p, sizeof(double));
  add(blk, sizeof(double));
  add(blk, sizeof(int));
  add(max_groups + 1, sizeof(int));
  add(max_groups, sizeof(double));
  add(max_groups, sizeof(double));
  for (int i = 0; i < 9; ++i) add(max_K + 1, sizeof(double));
  for (int i = 0; i < 8; ++i) add(n, sizeof(double));
  add(4, sizeof(int));
  cudaError_t e = cudaMalloc(&P->arena, bytes);
  if (e != cudaSuccess) {
    free(P);
    return TF_ERR_NOMEM;
  }
  unsigned char* cur = P->arena;
  P->twx = carve<float2>(cur, nx);
  P->rotx = carve<float2>(cur, nx);
  P->twy = carve<float2>(cur, ny);
  P->roty = carve<float2>(cur, ny);
  P->w = carve<double>(cur, 2 * P->R + 1);
  P->X = carve<float>(cur, (size_t)ny * P->Pb);
  P->A = carve<double>(cur, (size_t)P->Qb * P->Pb);
  P->T = carve<double>(cur, (size_t)P->Qb * P->n_p);
  P->S = carve<double>(cur, blk);
  P->member = carve<int>(cur, blk);
  P->roff = carve<int>(cur, max_groups + 1);
  P->rq = carve<double>(cur, max_groups);
  P->rv = carve<double>(cur, max_groups);
  P->t = carve<double>(cur, max_K + 1);
  P->diag = carve<double>(cur, max_K + 1);
  P->off = carve<double>(cur, max_K + 1);
  P->rhs = carve<double>(cur, max_K + 1);
  P->a = carve<double>(cur, max_K + 1);
  P->cp = carve<double>(cur, max_K + 1);
  P->zz = carve<double>(cur, max_K + 1);
  P->za = carve<double>(cur, max_K + 1);
  P->zb = carve<double>(cur, max_K + 1);
  P->w0 = carve<double>(cur, n);
  P->w1 = carve<double>(cur, n);
  P->dd = carve<double>(cur, n);
  P->ss = carve<double>(cur, n);
  P->cq = carve<double>(cur, n);
  P->cv = carve<double>(cur, n);
  P->pq = carve<double>(cur, n);
  P->pv = carve<double>(cur, n);
  P->d_npeaks = carve<int>(cur, 4);
  for (int i = 0; i <= kKernels; ++i) {
    if (cudaEventCreate(&P->ev[i]) != cudaSuccess) {
      tf_spectrum_plan_destroy(P);
      return TF_ERR_CUDA;
    }
  }

  // tables (host FP64, rounded once)
  float2* ht = (float2*)malloc(sizeof(float2) * (size_t)(2 * nx + 2 * ny));
  double* hw = (double*)malloc(sizeof(double) * (2 * P->R + 1));
  if (!ht || !hw) {
    free(ht);
    free(hw);
    tf_spectrum_plan_destroy(P);
    return TF_ERR_NOMEM;
  }
  float2 *htwx = ht, *hrotx = htwx + nx, *htwy = hrotx + nx, *hroty = htwy + ny;
  host_tables(nx, htwx, hrotx);
  host_tables(ny, htwy, hroty);
  {
    double sum = 0.0;
    for (int d = -P->R; d <= P->R; ++d) {
      hw[d + P->R] = P->R ? exp(-(double)d * d / (2.0 * sp->sigma * sp->sigma)) : 1.0;
      sum += hw[d + P->R];
    }
    for (int d = 0; d <= 2 * P->R; ++d) hw[d] /= sum;
  }
  cudaStream_t st = P->stream;
  e = cudaMemcpyAsync(P->twx, htwx, sizeof(float2) * nx, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(P->rotx, hrotx, sizeof(float2) * nx, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(P->twy, htwy, sizeof(float2) * ny, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(P->roty, hroty, sizeof(float2) * ny, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(P->w, hw, sizeof(double) * (2 * P->R + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  free(ht);
  free(hw);
  if (e != cudaSuccess) {
    tf_spectrum_plan_destroy(P);
    return TF_ERR_CUDA;
  }

  // radial grouping: counting sort of the block's points by key
  int *cnt = nullptr, *koff = nullptr, *meta = nullptr;
  long long* rkey = nullptr;
  e = cudaMalloc(&cnt, sizeof(int) * nkeys);
  if (e == cudaSuccess) e = cudaMalloc(&koff, sizeof(int) * nkeys);
  if (e == cudaSuccess) e = cudaMalloc(&rkey, sizeof(long long) * (max_groups + 1));
  if (e == cudaSuccess) e = cudaMalloc(&meta, sizeof(int) * 2);
  int hmeta[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int) * nkeys, st);
  if (e == cudaSuccess) {
    const dim3 grid((P->n_p + 255) / 256, P->n_q);
    k_keys_count<<<grid, 256, 0, st>>>(P->n_p, P->n_q, P->ax, P->ay, P->keycut, cnt);
    k_keys_scan<<<1, kFitThreads, 0, st>>>(cnt, nkeys, koff, rkey, P->roff, meta);
    e = cudaMemsetAsync(cnt, 0, sizeof(int) * nkeys, st);
    if (e == cudaSuccess) {
      k_keys_fill<<<grid, 256, 0, st>>>(P->n_p, P->n_q, P->ax, P->ay, P->keycut, koff, cnt, P->member);
      e = cudaMemcpyAsync(hmeta, meta, sizeof(hmeta), cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    P->M = hmeta[0];
    P->npts = hmeta[1];
    if (P->M >= 1) {
      k_keys_order<<<(P->M + 255) / 256, 256, 0, st>>>(P->M, rkey, P->roff, P->member, P->scale, P->rq);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
  }
  cudaFree(cnt);
  cudaFree(koff);
  cudaFree(rkey);
  cudaFree(meta);
  if (e != cudaSuccess) {
    tf_spectrum_plan_destroy(P);
    return TF_ERR_CUDA;
  }
  if (P->M < 2) {  // the fit needs the origin and one more radius
    tf_spectrum_plan_destroy(P);
    return TF_ERR_ARG;
  }
  P->K = std::max(1, (P->M - 1 + sp->points_per_interval - 1) / sp->points_per_interval);

  // opt-in shared memory of the FFT blocks (padded 16 THREADS values)
  e = cudaFuncSetAttribute(k_dct_rows<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_smem(512));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_dct_cols<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_smem(512));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_dct_rows<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_smem(1024));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_dct_cols<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_smem(1024));
  if (e != cudaSuccess) {
    tf_spectrum_plan_destroy(P);
    return TF_ERR_CUDA;
  }
  *out = P;
  return TF_OK;
}

int tf_spectrum_plan_info(const tf_spectrum_plan* P, tf_spectrum_info* info) {
  if (!P || !info) return TF_ERR_ARG;
  memset(info, 0, sizeof(*info));
  info->n_p = P->n_p;
  info->n_q = P->n_q;
  info->n_radii = P->M;
  info->n_intervals = P->K;
  info->n_eval = P->sp.n_eval;
  return TF_OK;
}

int tf_spectrum_run(tf_spectrum_plan* P, const double* h, tf_spectrum_out* out, tf_spectrum_info* info) {
  if (!P || !h || !info) return TF_ERR_ARG;
  if (out && out->peak_cap > 0 && (!out->peak_q || !out->peak_value)) return TF_ERR_ARG;
  cudaStream_t st = P->stream;
  const int nx = P->nx, ny = P->ny;
  cudaError_t e = cudaSuccess;
  const int row_pairs = (ny + 1) / 2, col_pairs = (P->Pb + 1) / 2;
  const int Gx = 16 * P->thx / nx, Gy = 16 * P->thy / ny;
  const dim3 grow((row_pairs + Gx - 1) / Gx), gcol((col_pairs + Gy - 1) / Gy);
  const double inv = 1.0 / ((double)nx * ny);
  cudaEventRecord(P->ev[0], st);
  const double H0 = P->sp.H0;
  const float H0hi = (float)H0, H0lo = (float)(H0 - (double)H0hi);
  if (P->thx == 512)
    k_dct_rows<512><<<grow, 512, fft_smem(512), st>>>(h, nx, ny, H0, H0hi, H0lo, P->lgx, P->Pb, P->twx, P->rotx,
                                                        P->X);
  else
    k_dct_rows<1024><<<grow, 1024, fft_smem(1024), st>>>(h, nx, ny, H0, H0hi, H0lo, P->lgx, P->Pb, P->twx,
                                                          P->rotx, P->X);
  cudaEventRecord(P->ev[1], st);
  if (P->thy == 512)
    k_dct_cols<512><<<gcol, 512, fft_smem(512), st>>>(P->X, ny, P->Pb, P->Qb, P->lgy, P->twy, P->roty, inv, P->A);
  else
    k_dct_cols<1024><<<gcol, 1024, fft_smem(1024), st>>>(P->X, ny, P->Pb, P->Qb, P->lgy, P->twy, P->roty, inv, P->A);
  cudaEventRecord(P->ev[2], st);
  k_smooth_p<<<dim3((P->n_p + 127) / 128, P->Qb), 128, 0, st>>>(P->A, P->Pb, P->Qb, P->n_p, nx, P->R, P->w, P->T);
  cudaEventRecord(P->ev[3], st);
  k_smooth_q<<<dim3((P->n_p + 127) / 128, P->n_q), 128, 0, st>>>(P->T, P->n_p, P->n_q, ny, P->R, P->w, P->S);
  cudaEventRecord(P->ev[4], st);
  k_radial_mean<<<(P->M + 255) / 256, 256, 0, st>>>(P->M, P->roff, P->member, P->S, P->rv);
  cudaEventRecord(P->ev[5], st);
  FitArgs f;
  f.M = P->M;
  f.K = P->K;
  f.ppi = P->sp.points_per_interval;
  f.n_eval = P->sp.n_eval;
  f.q_cut = P->sp.q_cut;
  f.rq = P->rq;
  f.rv = P->rv;
  f.t = P->t;
  f.diag = P->diag;
  f.off = P->off;
  f.rhs = P->rhs;
  f.a = P->a;
  f.cp = P->cp;
  f.zz = P->zz;
  f.za = P->za;
  f.zb = P->zb;
  f.w0 = P->w0;
  f.w1 = P->w1;
  f.d = P->dd;
  f.s = P->ss;
  f.cq = P->cq;
  f.cv = P->cv;
  f.pq = P->pq;
  f.pv = P->pv;
  f.n_peaks = P->d_npeaks;
  {
    const int c = fit_chunk(P->K), S = P->K / c;
    k_fit_assemble<<<(P->K + 63) / 64, 64, 0, st>>>(f);
    k_fit_blocks<<<(S + 1 + 31) / 32, 32, 0, st>>>(f);
    k_fit_reduced<<<1, kReduced, 0, st>>>(f);
    k_fit_back<<<(P->K + 127) / 128, 128, 0, st>>>(f);
    k_fit_peaks<<<1, kFitThreads, 0, st>>>(f);
  }
  cudaEventRecord(P->ev[6], st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return TF_ERR_CUDA;

  int np = 0;
  double top[2] = {0.0, 0.0};
  e = cudaMemcpyAsync(&np, P->d_npeaks, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return TF_ERR_CUDA;
  if (np > 0) {
    e = cudaMemcpyAsync(&top[0], P->pq, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&top[1], P->pv, sizeof(double), cudaMemcpyDeviceToHost, st);
  }
  const size_t blk = (size_t)P->n_p * P->n_q;
  auto fetch = [&](double* dst, const double* src, size_t cnt) {
    if (e == cudaSuccess && dst && cnt) e = cudaMemcpyAsync(dst, src, cnt * sizeof(double), cudaMemcpyDeviceToHost, st);
  };
  auto fetch2d = [&](double* dst, const double* src, size_t pitch) {
    if (e == cudaSuccess && dst)
      e = cudaMemcpy2DAsync(dst, sizeof(double) * P->n_p, src, sizeof(double) * pitch, sizeof(double) * P->n_p,
                            P->n_q, cudaMemcpyDeviceToHost, st);
  };
  if (out) {
    fetch2d(out->amplitude, P->A, P->Pb);
    fetch(out->smoothed, P->S, blk);
    fetch(out->radial_q, P->rq, P->M);
    fetch(out->radial_value, P->rv, P->M);
    fetch(out->node_q, P->t, P->K + 1);
    fetch(out->node_value, P->a, P->K + 1);
    fetch(out->curve_q, P->cq, P->sp.n_eval);
    fetch(out->curve_value, P->cv, P->sp.n_eval);
    const int cp = std::min(np, out->peak_cap);
    fetch(out->peak_q, P->pq, cp);
    fetch(out->peak_value, P->pv, cp);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return TF_ERR_CUDA;
  for (int k = 0; k < kKernels; ++k) cudaEventElapsedTime(&P->ms[k], P->ev[k], P->ev[k + 1]);
  tf_spectrum_plan_info(P, info);
  info->n_peaks = np;
  info->q_dominant = top[0];
  info->value_dominant = top[1];
  return TF_OK;
}

int tf_spectrum_timing(const tf_spectrum_plan* P, double* ms, int n) {
  if (!P || !ms || n < 1) return TF_ERR_ARG;
  for (int k = 0; k < n && k < kKernels; ++k) ms[k] = P->ms[k];
  return TF_OK;
}

}  // extern "C"
