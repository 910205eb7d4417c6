// SE(3) exponential with one tangent direction (X-SLAM Sec. 4.1, Eq. lie, rotvector, rotation_jacobi)
// for the pose update T <- exp(x) T of ICP, evaluated one matrix element per thread. The ICP step x is
// small, so the update is formed as exp(x) = I + delta with delta computed in FP32 (its relative
// precision is what matters) and T <- T + delta T composed in FP64. The FP64 variants also serve the
// host (xslam_se3_exp_compose).
//
// exp([phi, rho]) = [R | V rho] with R = I + A [phi] + B [phi]^2 and V = I + B [phi] + C [phi]^2,
// A = sin(th)/th, B = (1 - cos th)/th^2, C = (th - sin th)/th^3, th^2 = phi.phi; this is the
// paper's cos/sin/axis form rewritten with [a]^2 = a a^T - I so that it has no 1/th at th = 0. A, B,
// C are evaluated as power series in th^2 below th^2 = 1/4 (exact limits, no cancellation) and in
// closed form above. The tangent (imaginary lane) follows by differentiating A, B, C in th^2.
#pragma once

namespace xslam {

struct Coef {
  double A, B, C, dA, dB, dC;  // values and derivatives with respect to x = th^2
};

// sum_{n=0}^{N} (-x)^n / (2n+1+s)! and its derivative in x by Horner's rule (s = 0: A, 1: B, 2: C)
template <int N>
__host__ __device__ __forceinline__ void series(double x, int s, double& v, double& dv) {
  constexpr double inv_fact[22] = {
      1.0, 1.0, 1.0 / 2.0, 1.0 / 6.0, 1.0 / 24.0, 1.0 / 120.0, 1.0 / 720.0, 1.0 / 5040.0, 1.0 / 40320.0,
      1.0 / 362880.0, 1.0 / 3628800.0, 1.0 / 39916800.0, 1.0 / 479001600.0, 1.0 / 6227020800.0,
      1.0 / 87178291200.0, 1.0 / 1307674368000.0, 1.0 / 20922789888000.0, 1.0 / 355687428096000.0,
      1.0 / 6402373705728000.0, 1.0 / 121645100408832000.0, 1.0 / 2432902008176640000.0,
      1.0 / 51090942171709440000.0};
  v = ((N & 1) ? -1.0 : 1.0) * inv_fact[2 * N + 1 + s];
  dv = 0.0;
#pragma unroll
  for (int n = N - 1; n >= 0; --n) {
    dv = dv * x + v;
    v = v * x + ((n & 1) ? -1.0 : 1.0) * inv_fact[2 * n + 1 + s];
  }
}

__host__ __device__ __forceinline__ Coef se3_coef(double x) {
  Coef c;
  if (x < 1e-2) {
    // terms up to x^5: truncation below 2e-22 for x < 1e-2 (rotations under 0.1 rad, every ICP step)
    series<5>(x, 0, c.A, c.dA);
    series<5>(x, 1, c.B, c.dB);
    series<5>(x, 2, c.C, c.dC);
  } else if (x < 0.25) {
    // terms up to x^9: truncation below 1e-25 for x < 1/4
    series<9>(x, 0, c.A, c.dA);
    series<9>(x, 1, c.B, c.dB);
    series<9>(x, 2, c.C, c.dC);
  } else {
    const double th = sqrt(x), s = sin(th), co = cos(th);
    c.A = s / th;
    c.B = (1.0 - co) / x;
    c.C = (th - s) / (x * th);
    c.dA = (th * co - s) / (2.0 * x * th);
    c.dB = (th * s - 2.0 * (1.0 - co)) / (2.0 * x * x);
    c.dC = ((1.0 - co) * th - 3.0 * (th - s)) / (2.0 * x * x * th);
  }
  return c;
}

// Coefficients of exp at x0 and the tangent of theta^2 along x1 (one per lane, shared by its elements).
struct SeCoef {
  double A, B, C, dA, dB, dC;  // dA etc.: tangents along x1 (derivative in theta^2 times d theta^2)
};

__host__ __device__ __forceinline__ void se3_coef_lane(const double* x0, const double* x1, SeCoef& out) {
  const double th2 = x0[0] * x0[0] + x0[1] * x0[1] + x0[2] * x0[2];
  const double dth2 = 2.0 * (x0[0] * x1[0] + x0[1] * x1[1] + x0[2] * x1[2]);
  const Coef c = se3_coef(th2);
  out.A = c.A;
  out.B = c.B;
  out.C = c.C;
  out.dA = c.dA * dth2;
  out.dB = c.dB * dth2;
  out.dC = c.dC * dth2;
}

// [v]_{rk}
__host__ __device__ __forceinline__ double hat_el(const double* v, int r, int k) {
  if (r == k) return 0.0;
  if (r == 0) return k == 1 ? -v[2] : v[1];
  if (r == 1) return k == 0 ? v[2] : -v[0];
  return k == 0 ? -v[1] : v[0];
}

// ([phi]^2)_{rk} = phi_r phi_k - th2 delta_rk and its tangent along phi1
__host__ __device__ __forceinline__ double hat2_el(const double* v, int r, int k) {
  return v[r] * v[k] - (r == k ? v[0] * v[0] + v[1] * v[1] + v[2] * v[2] : 0.0);
}
__host__ __device__ __forceinline__ double hat2_tan(const double* v, const double* v1, int r, int k) {
  return v1[r] * v[k] + v[r] * v1[k] - (r == k ? 2.0 * (v[0] * v1[0] + v[1] * v1[1] + v[2] * v1[2]) : 0.0);
}

// Element e = 4 r + c of E = exp(x0) (tangent = false) or of its tangent along x1 (tangent = true).
__host__ __device__ __forceinline__ double se3_exp_element(const double* x0, const double* x1, const SeCoef& k, bool tangent,
                                                  int e) {
  const int r = e >> 2, c = e & 3;
  if (c < 3) {
    if (!tangent) return (r == c ? 1.0 : 0.0) + k.A * hat_el(x0, r, c) + k.B * hat2_el(x0, r, c);
    return k.dA * hat_el(x0, r, c) + k.A * hat_el(x1, r, c) + k.dB * hat2_el(x0, r, c) + k.B * hat2_tan(x0, x1, r, c);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const double V = (r == q ? 1.0 : 0.0) + k.B * hat_el(x0, r, q) + k.C * hat2_el(x0, r, q);
    if (!tangent) {
      s += V * x0[3 + q];
    } else {
      const double V1 = k.dB * hat_el(x0, r, q) + k.B * hat_el(x1, r, q) + k.dC * hat2_el(x0, r, q) +
                        k.C * hat2_tan(x0, x1, r, q);
      s += V1 * x0[3 + q] + V * x1[3 + q];
    }
  }
  return s;
}

// ---- FP32 increment: delta = exp(x) - I for the small ICP step x, composed in FP64 by the caller ----
// A, B, C of exp and their tangents in FP32 (series for theta^2 < 1/4, closed form above)
struct SeCoefF {
  float A, B, C, dA, dB, dC;
};

template <int N>
__device__ __forceinline__ void series_f(float x, int s, float& v, float& dv) {
  constexpr float inv_fact[16] = {1.f, 1.f, 1.f / 2, 1.f / 6, 1.f / 24, 1.f / 120, 1.f / 720, 1.f / 5040,
                                  1.f / 40320, 1.f / 362880, 1.f / 3628800, 1.f / 39916800, 1.f / 479001600,
                                  1.f / 6227020800.f, 1.f / 87178291200.f, 1.f / 1307674368000.f};
  v = ((N & 1) ? -1.f : 1.f) * inv_fact[2 * N + 1 + s];
  dv = 0.f;
#pragma unroll
  for (int n = N - 1; n >= 0; --n) {
    dv = dv * x + v;
    v = v * x + ((n & 1) ? -1.f : 1.f) * inv_fact[2 * n + 1 + s];
  }
}

__device__ __forceinline__ void se3_coef_lane_f(const float* x0, const float* x1, SeCoefF& out) {
  const float th2 = x0[0] * x0[0] + x0[1] * x0[1] + x0[2] * x0[2];
  const float dth2 = 2.f * (x0[0] * x1[0] + x0[1] * x1[1] + x0[2] * x1[2]);
  float A, B, C, dA, dB, dC;
  if (th2 < 0.25f) {  // terms up to x^6: truncation below 2e-12 relative for x < 1/4
    series_f<6>(th2, 0, A, dA);
    series_f<6>(th2, 1, B, dB);
    series_f<6>(th2, 2, C, dC);
  } else {
    const float th = sqrtf(th2), s = sinf(th), co = cosf(th);
    A = s / th;
    B = (1.f - co) / th2;
    C = (th - s) / (th2 * th);
    dA = (th * co - s) / (2.f * th2 * th);
    dB = (th * s - 2.f * (1.f - co)) / (2.f * th2 * th2);
    dC = ((1.f - co) * th - 3.f * (th - s)) / (2.f * th2 * th2 * th);
  }
  out.A = A;
  out.B = B;
  out.C = C;
  out.dA = dA * dth2;
  out.dB = dB * dth2;
  out.dC = dC * dth2;
}

__device__ __forceinline__ float hat_el_f(const float* v, int r, int k) {
  if (r == k) return 0.f;
  if (r == 0) return k == 1 ? -v[2] : v[1];
  if (r == 1) return k == 0 ? v[2] : -v[0];
  return k == 0 ? -v[1] : v[0];
}
__device__ __forceinline__ float hat2_el_f(const float* v, int r, int k) {
  return v[r] * v[k] - (r == k ? v[0] * v[0] + v[1] * v[1] + v[2] * v[2] : 0.f);
}
__device__ __forceinline__ float hat2_tan_f(const float* v, const float* v1, int r, int k) {
  return v1[r] * v[k] + v[r] * v1[k] - (r == k ? 2.f * (v[0] * v1[0] + v[1] * v1[1] + v[2] * v1[2]) : 0.f);
}

// Element e = 4 r + c of exp(x0) - I (tangent = false) or of the tangent of exp along x1 (true).
__device__ __forceinline__ float se3_delta_element(const float* x0, const float* x1, const SeCoefF& k, bool tangent,
                                                   int e) {
  const int r = e >> 2, c = e & 3;
  if (c < 3) {
    if (!tangent) return k.A * hat_el_f(x0, r, c) + k.B * hat2_el_f(x0, r, c);
    return k.dA * hat_el_f(x0, r, c) + k.A * hat_el_f(x1, r, c) + k.dB * hat2_el_f(x0, r, c) +
           k.B * hat2_tan_f(x0, x1, r, c);
  }
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const float V = (r == q ? 1.f : 0.f) + k.B * hat_el_f(x0, r, q) + k.C * hat2_el_f(x0, r, q);
    if (!tangent) {
      s += V * x0[3 + q];
    } else {
      const float V1 = k.dB * hat_el_f(x0, r, q) + k.B * hat_el_f(x1, r, q) + k.dC * hat2_el_f(x0, r, q) +
                       k.C * hat2_tan_f(x0, x1, r, q);
      s += V1 * x0[3 + q] + V * x1[3 + q];
    }
  }
  return s;
}

}  // namespace xslam
