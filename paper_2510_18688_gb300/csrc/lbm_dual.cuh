// lbm_dual.cuh -- forward-mode (tangent) arithmetic for the step kernels.
//
// A Dual carries a double value and its derivative along one direction of
// the parameters (dual numbers: (a, a')(b, b') = (ab, a'b + ab'), and so
// on).  Instantiating the step template with Dual computes, in the same
// launch and with the same branch decisions as the FP64 step, the
// derivative of every population, lag field and diagnostic with respect to
// the chosen parameter direction.  Comparisons look at the value only, so
// at the kinks of the enthalpy inversion (Eq. (8)) and of the clamps the
// derivative is the one of the branch taken.
#pragma once

#include <cmath>
#include <type_traits>

#include <cuda_runtime.h>

namespace lbmk {

struct Dual {
  double v, d;
  Dual() = default;  // trivial, as double: shared-memory arrays of it are allowed
  __host__ __device__ constexpr Dual(double x) : v(x), d(0.0) {}  // NOLINT: a constant
  __host__ __device__ constexpr Dual(double x, double dx) : v(x), d(dx) {}
  __host__ __device__ Dual& operator+=(const Dual& b) { v += b.v; d += b.d; return *this; }
  __host__ __device__ Dual& operator-=(const Dual& b) { v -= b.v; d -= b.d; return *this; }
  __host__ __device__ Dual& operator*=(const Dual& b) {
    d = d * b.v + v * b.d;
    v *= b.v;
    return *this;
  }
};

__host__ __device__ inline Dual operator+(Dual a, const Dual& b) { return a += b; }
__host__ __device__ inline Dual operator-(Dual a, const Dual& b) { return a -= b; }
__host__ __device__ inline Dual operator*(Dual a, const Dual& b) { return a *= b; }
__host__ __device__ inline Dual operator-(const Dual& a) { return Dual(-a.v, -a.d); }
__host__ __device__ inline Dual operator/(const Dual& a, const Dual& b) {
  const double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
__host__ __device__ inline bool operator<(const Dual& a, const Dual& b) { return a.v < b.v; }
__host__ __device__ inline bool operator>(const Dual& a, const Dual& b) { return a.v > b.v; }
__host__ __device__ inline bool operator<=(const Dual& a, const Dual& b) { return a.v <= b.v; }
__host__ __device__ inline bool operator>=(const Dual& a, const Dual& b) { return a.v >= b.v; }

template <typename R>
struct is_dual : std::false_type {};
template <>
struct is_dual<Dual> : std::true_type {};

__device__ __forceinline__ Dual qdiv(const Dual& a, const Dual& b) { return a / b; }
// finite(): value and derivative both finite (plain types: the usual test)
__device__ __forceinline__ bool finite(float a) { return ::isfinite(a); }
__device__ __forceinline__ bool finite(double a) { return ::isfinite(a); }
__device__ __forceinline__ bool finite(const Dual& a) { return ::isfinite(a.v) && ::isfinite(a.d); }
__device__ __forceinline__ Dual ldp(const Dual* p) { return *p; }
__device__ __forceinline__ void stp(Dual* p, const Dual& x) { *p = x; }
__device__ __forceinline__ Dual shfl_xor(const Dual& x, int o) {
  return Dual(__shfl_xor_sync(0xffffffffu, x.v, o), __shfl_xor_sync(0xffffffffu, x.d, o));
}

}  // namespace lbmk
