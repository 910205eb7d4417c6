// Bicomplex numbers in FP64 for the plain comparison paths: Sec. 3's second-order step as printed.
// A number a + b i1 + c i2 + d i1 i2 with i1^2 = i2^2 = -1 and i1 i2 = i2 i1; every product is kept.
// With a step h folded into the start poses (b, c scaled by h, d by h^2), the i1 and i2 parts of a
// result are h times its first derivatives along the two directions and the i1 i2 part is h^2 times the
// mixed second derivative (exact to O(h^2) relative; h = 1e-20 leaves no truncation error in FP64).
#pragma once

#include <cuda_runtime.h>

namespace xslam {

struct BC {
  double a, b, c, d;
};
__device__ __forceinline__ BC bc(double a) { return {a, 0.0, 0.0, 0.0}; }
__device__ __forceinline__ BC operator+(BC x, BC y) { return {x.a + y.a, x.b + y.b, x.c + y.c, x.d + y.d}; }
__device__ __forceinline__ BC operator-(BC x, BC y) { return {x.a - y.a, x.b - y.b, x.c - y.c, x.d - y.d}; }
__device__ __forceinline__ BC operator+(BC x, double s) { return {x.a + s, x.b, x.c, x.d}; }
__device__ __forceinline__ BC operator*(double s, BC x) { return {s * x.a, s * x.b, s * x.c, s * x.d}; }
__device__ __forceinline__ BC operator*(BC x, BC y) {
  return {x.a * y.a - x.b * y.b - x.c * y.c + x.d * y.d, x.a * y.b + x.b * y.a - x.c * y.d - x.d * y.c,
          x.a * y.c + x.c * y.a - x.b * y.d - x.d * y.b, x.a * y.d + x.d * y.a + x.b * y.c + x.c * y.b};
}
// 1/z: with z = z1 + z2 i2 (z1 = a + b i1, z2 = c + d i1 complex in i1), 1/z = (z1 - z2 i2) / (z1^2 + z2^2)
__device__ __forceinline__ BC binv(BC z) {
  const double p = z.a * z.a - z.b * z.b + z.c * z.c - z.d * z.d, q = 2.0 * (z.a * z.b + z.c * z.d);
  const double n = p * p + q * q, r = p / n, s = -q / n;  // 1/(p + q i1) = r + s i1
  return {z.a * r - z.b * s, z.a * s + z.b * r, -(z.c * r - z.d * s), -(z.c * s + z.d * r)};
}
// Principal square root of a number with a > 0 whose other parts are O(h): the analytic function on
// z = z1 + z2 i2 taken as f(z1) + f'(z1) z2 i2, each complex-in-i1 factor likewise (the parts of order
// h^2 and above that reach a, b or c are below FP64 rounding): with s = sqrt(a), s' = 1 / (2 s),
// s'' = -1 / (4 s a): sqrt(z) = s + s' b i1 + s' c i2 + (s' d + s'' b c) i1 i2.
__device__ __forceinline__ BC bsqrt(BC z) {
  const double s = sqrt(z.a), s1 = 0.5 / s, s2 = -0.25 / (s * z.a);
  return {s, s1 * z.b, s1 * z.c, s1 * z.d + s2 * z.b * z.c};
}

}  // namespace xslam
