// Reciprocal square root and quotient for the push's Boris step (device code, header only).
#pragma once

namespace picgb {

__device__ __forceinline__ float fast_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ float fast_div(float a, float b) { return __fdividef(a, b); }
// FP64: Newton-Raphson refinement of an FP32 estimate instead of the IEEE FP64 square root and
// division, which are long instruction sequences on the FP64 pipe that bounds this kernel. Each
// step squares the relative error (an FP32 estimate's ~1e-7, then ~1e-14), so two steps reach the
// FP64 rounding level; the quotient adds one residual correction (Markstein's scheme: q + (a - b q) y).
// The arguments are the Boris step's 1 + u^2, 1 + t^2 and gamma + 1: positive and finite (a NaN or
// infinite one comes out NaN, which the non-finite check after the move catches).
__device__ __forceinline__ double fast_rsqrt(double x) {
  double y = (double)rsqrtf((float)x);
  const double h = 0.5 * x;
  y = y * fma(-h * y, y, 1.5);  // y (3 - x y^2) / 2
  y = y * fma(-h * y, y, 1.5);
  return y;
}
__device__ __forceinline__ double fast_div(double a, double b) {
  double y = (double)__fdividef(1.f, (float)b);
  y = fma(fma(-b, y, 1.0), y, y);  // y (2 - b y)
  y = fma(fma(-b, y, 1.0), y, y);
  const double q = a * y;
  return fma(fma(-b, q, a), y, q);
}

}  // namespace picgb
