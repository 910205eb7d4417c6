// Truncated bicomplex numbers a + b e1 + c e2 + d e1 e2 with e1^2 = e2^2 = 0: the simplified
// arithmetic of X-SLAM Sec. 3 (products of two perturbations of the same unit dropped) carrying a value,
// its derivatives along two directions and the mixed second derivative (the e1 e2 part) exactly. Shared
// by the relocalisation Hessian (hess.cu) and Newton ICP (icp_newton.cu).
#pragma once

namespace xslam {

struct HD {
  float a, b, c, d;
};
__device__ __forceinline__ HD hd(float a) { return {a, 0.f, 0.f, 0.f}; }
__device__ __forceinline__ HD operator+(HD x, HD y) { return {x.a + y.a, x.b + y.b, x.c + y.c, x.d + y.d}; }
__device__ __forceinline__ HD operator-(HD x, HD y) { return {x.a - y.a, x.b - y.b, x.c - y.c, x.d - y.d}; }
__device__ __forceinline__ HD operator+(HD x, float s) { return {x.a + s, x.b, x.c, x.d}; }
__device__ __forceinline__ HD operator*(float s, HD x) { return {s * x.a, s * x.b, s * x.c, s * x.d}; }
__device__ __forceinline__ HD operator*(HD x, HD y) {
  return {x.a * y.a, x.a * y.b + x.b * y.a, x.a * y.c + x.c * y.a, x.a * y.d + x.d * y.a + x.b * y.c + x.c * y.b};
}
// 1/y: f = 1/a, f' = -1/a^2, f'' = 2/a^3 (f(a + t) = f + f' t + f'' t^2 / 2, t^2 = 2 b c e1 e2)
__device__ __forceinline__ HD inv(HD y) {
  const float r = 1.f / y.a, r2 = r * r;
  return {r, -r2 * y.b, -r2 * y.c, -r2 * y.d + 2.f * r2 * r * y.b * y.c};
}
__device__ __forceinline__ HD operator/(HD x, HD y) { return x * inv(y); }
// sqrt: f' = 1/(2 s), f'' = -1/(4 s^3)
__device__ __forceinline__ HD hsqrt(HD y) {
  const float s = sqrtf(y.a), r = 0.5f / s;
  return {s, r * y.b, r * y.c, r * y.d - 0.25f * y.b * y.c / (s * s * s)};
}

}  // namespace xslam
