// Host build of the numeric layer (tf_numeric.cuh) for the CPU unit tests:
// the same source the kernels use, exported with plain C entry points.
#include "tf_numeric.cuh"

extern "C" {
void tfh_f32_trunc_of_f64(const double* x, float* y, long n) {
  for (long i = 0; i < n; ++i) y[i] = tf::f32_trunc_of_f64(x[i]);
}
void tfh_df_of_f64(const double* x, float* hi, float* lo, long n) {
  for (long i = 0; i < n; ++i) {
    tf::df64 d = tf::df_of_f64(x[i]);
    hi[i] = d.hi;
    lo[i] = d.lo;
  }
}
void tfh_f64_add_f32(const double* u, const float* v, double* y, long n) {
  for (long i = 0; i < n; ++i) y[i] = tf::f64_add_f32(u[i], v[i]);
}
void tfh_df_ops(const double* a, const double* b, double* sum, double* prod, double* rcp, long n) {
  for (long i = 0; i < n; ++i) {
    tf::df64 x = tf::df_of_f64(a[i]), y = tf::df_of_f64(b[i]);
    sum[i] = tf::f64_of_df(x - y);
    prod[i] = tf::f64_of_df(x * y);
    rcp[i] = tf::f64_of_df(tf::df_rcp(x));
  }
}
void tfh_fast_conv(const double* x, float* f, float* hi, float* lo, long n) {
  for (long i = 0; i < n; ++i) {
    f[i] = tf::f32_of_pos_f64_fast(x[i]);
    tf::df64 d = tf::df_of_pos_f64_fast(x[i]);
    hi[i] = d.hi;
    lo[i] = d.lo;
  }
}
// bit patterns b in [lo, hi) whose float f64_of_f32_exact widens to other
// bits than the host's own float -> double conversion
long tfh_f64_of_f32_exact_mismatches(unsigned long long lo, unsigned long long hi) {
  long bad = 0;
  for (unsigned long long b = lo; b < hi; ++b) {
    const float f = tf::float_of((uint32_t)b);
    const double w = tf::f64_of_f32_exact(f), r = (double)f;
    if (tf::bits_of(w) != tf::bits_of(r)) ++bad;
  }
  return bad;
}
void tfh_f64_of_f32_exact(const float* x, double* y, long n) {
  for (long i = 0; i < n; ++i) y[i] = tf::f64_of_f32_exact(x[i]);
}
void tfh_fixed36(const double* u, long long* q, long n) {
  for (long i = 0; i < n; ++i) q[i] = (long long)tf::fixed36_of_f64(u[i]);
}
}
