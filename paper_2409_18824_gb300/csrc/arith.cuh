// Separately rounded adds and multiplies for the canonical evaluation order.
//
// The double path issues every add as fma(a, 1, b) and every multiply as
// fma(a, b, -0): both round exactly like a plain add / multiply (a*1 and the
// -0 addend are exact, and -0 keeps the sign of a zero product), but they go
// through the FMA issue path, which sustains 2 double ops/clk/SM on this GPU
// against 1.7 for plain adds.  They are written as inline PTX so that the
// compiler cannot fold them back into add/mul and then contract a multiply
// and a following add into one fused operation, which would change rounding.
#pragma once

namespace stn {

template <typename T>
struct Arith;

template <>
struct Arith<double> {
  static __device__ __forceinline__ double add(double a, double b) {
    double r;
    asm("fma.rn.f64 %0, %1, 0d3FF0000000000000, %2;" : "=d"(r) : "d"(a), "d"(b));
    return r;
  }
  static __device__ __forceinline__ double mul(double a, double b) {
    double r;
    asm("fma.rn.f64 %0, %1, %2, 0d8000000000000000;" : "=d"(r) : "d"(a), "d"(b));
    return r;
  }
  static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
};

template <>
struct Arith<float> {
  static __device__ __forceinline__ float add(float a, float b) {
    float r;
    asm("add.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
  }
  static __device__ __forceinline__ float mul(float a, float b) {
    float r;
    asm("mul.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
  }
  static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
};

}  // namespace stn
