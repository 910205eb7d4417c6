// FP64 SE(3) exponential with one tangent direction (X-SLAM Sec. 4.1, Eq. lie, rotvector,
// rotation_jacobi), for the pose update T <- exp(x) T of ICP and the POSE0 seed.
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

// sum_{n=0}^{9} (-x)^n / (2n+1+s)! and its derivative in x by Horner's rule (s = 0: A, 1: B, 2: C)
__device__ __forceinline__ void series(double x, int s, double& v, double& dv) {
  constexpr double inv_fact[22] = {
      1.0, 1.0, 1.0 / 2.0, 1.0 / 6.0, 1.0 / 24.0, 1.0 / 120.0, 1.0 / 720.0, 1.0 / 5040.0, 1.0 / 40320.0,
      1.0 / 362880.0, 1.0 / 3628800.0, 1.0 / 39916800.0, 1.0 / 479001600.0, 1.0 / 6227020800.0,
      1.0 / 87178291200.0, 1.0 / 1307674368000.0, 1.0 / 20922789888000.0, 1.0 / 355687428096000.0,
      1.0 / 6402373705728000.0, 1.0 / 121645100408832000.0, 1.0 / 2432902008176640000.0,
      1.0 / 51090942171709440000.0};
  constexpr int N = 9;
  v = ((N & 1) ? -1.0 : 1.0) * inv_fact[2 * N + 1 + s];
  dv = 0.0;
#pragma unroll
  for (int n = N - 1; n >= 0; --n) {
    dv = dv * x + v;
    v = v * x + ((n & 1) ? -1.0 : 1.0) * inv_fact[2 * n + 1 + s];
  }
}

__device__ __forceinline__ Coef se3_coef(double x) {
  Coef c;
  if (x < 0.25) {
    // power series (terms up to x^9: truncation below 1e-25 for x < 1/4)
    series(x, 0, c.A, c.dA);
    series(x, 1, c.B, c.dB);
    series(x, 2, c.C, c.dC);
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

// E = exp(x0) and its tangent E1 along x1 (both 3x4 row-major). x1 == nullptr: tangent not wanted.
__device__ inline void se3_exp_tangent(const double* x0, const double* x1, double* E, double* E1) {
  const double p0 = x0[0], p1 = x0[1], p2 = x0[2];
  const double th2 = p0 * p0 + p1 * p1 + p2 * p2;
  const Coef c = se3_coef(th2);
  // [phi] and [phi]^2 = phi phi^T - th2 I
  const double H[9] = {0, -p2, p1, p2, 0, -p0, -p1, p0, 0};
  const double phi[3] = {p0, p1, p2};
  double H2[9];
  for (int r = 0; r < 3; ++r)
    for (int q = 0; q < 3; ++q) H2[3 * r + q] = phi[r] * phi[q] - (r == q ? th2 : 0.0);
  double R[9], Vm[9];
  for (int i = 0; i < 9; ++i) {
    const double I = (i % 4 == 0) ? 1.0 : 0.0;
    R[i] = I + c.A * H[i] + c.B * H2[i];
    Vm[i] = I + c.B * H[i] + c.C * H2[i];
  }
  for (int r = 0; r < 3; ++r) {
    E[4 * r + 0] = R[3 * r + 0];
    E[4 * r + 1] = R[3 * r + 1];
    E[4 * r + 2] = R[3 * r + 2];
    E[4 * r + 3] = Vm[3 * r] * x0[3] + Vm[3 * r + 1] * x0[4] + Vm[3 * r + 2] * x0[5];
  }
  if (!x1) return;
  const double q0 = x1[0], q1 = x1[1], q2 = x1[2];
  const double dth2 = 2.0 * (p0 * q0 + p1 * q1 + p2 * q2);
  const double Hd[9] = {0, -q2, q1, q2, 0, -q0, -q1, q0, 0};
  const double phd[3] = {q0, q1, q2};
  double H2d[9];
  for (int r = 0; r < 3; ++r)
    for (int q = 0; q < 3; ++q) H2d[3 * r + q] = phd[r] * phi[q] + phi[r] * phd[q] - (r == q ? dth2 : 0.0);
  const double dA = c.dA * dth2, dB = c.dB * dth2, dC = c.dC * dth2;
  double Rd[9], Vd[9];
  for (int i = 0; i < 9; ++i) {
    Rd[i] = dA * H[i] + c.A * Hd[i] + dB * H2[i] + c.B * H2d[i];
    Vd[i] = dB * H[i] + c.B * Hd[i] + dC * H2[i] + c.C * H2d[i];
  }
  for (int r = 0; r < 3; ++r) {
    E1[4 * r + 0] = Rd[3 * r + 0];
    E1[4 * r + 1] = Rd[3 * r + 1];
    E1[4 * r + 2] = Rd[3 * r + 2];
    E1[4 * r + 3] = Vd[3 * r] * x0[3] + Vd[3 * r + 1] * x0[4] + Vd[3 * r + 2] * x0[5] + Vm[3 * r] * x1[3] +
                    Vm[3 * r + 1] * x1[4] + Vm[3 * r + 2] * x1[5];
  }
}

// C = A * B for 3x4 rigid transforms.
__device__ __forceinline__ void compose(const double* A, const double* B, double* C) {
  for (int r = 0; r < 3; ++r) {
    for (int q = 0; q < 4; ++q) {
      double s = A[4 * r] * B[q] + A[4 * r + 1] * B[4 + q] + A[4 * r + 2] * B[8 + q];
      if (q == 3) s += A[4 * r + 3];
      C[4 * r + q] = s;
    }
  }
}

// Tangent of A * B: A1 * B + A * B1 (translation column without A's own translation term twice).
__device__ __forceinline__ void compose_tangent(const double* A, const double* A1, const double* B, const double* B1,
                                                double* C1) {
  for (int r = 0; r < 3; ++r) {
    for (int q = 0; q < 4; ++q) {
      double s = A1[4 * r] * B[q] + A1[4 * r + 1] * B[4 + q] + A1[4 * r + 2] * B[8 + q];
      s += A[4 * r] * B1[q] + A[4 * r + 1] * B1[4 + q] + A[4 * r + 2] * B1[8 + q];
      if (q == 3) s += A1[4 * r + 3];
      C1[4 * r + q] = s;
    }
  }
}

}  // namespace xslam
