// Scalar types and model constants shared by the device code and the host
// operation-count tool: the forward-mode Dual number, sincos for plain and
// dual scalars, and the quadrotor constants.  Compiles as CUDA or as plain C++
// (the host tool instantiates the model with a counting scalar).
#pragma once

#include <math.h>

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace bipm {

// ------------------------------------------------------------------ dual numbers
// Forward-mode scalar (value, one directional derivative).  Running the RK4
// adjoint with these scalars gives Hessian-vector products of lambda^T F
// (forward-over-reverse differentiation).
template <class T>
struct Dual {
  T v, d;
};

template <class T> __host__ __device__ __forceinline__ Dual<T> mk(T v, T d) { return Dual<T>{v, d}; }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator+(Dual<T> a, Dual<T> b) { return {a.v + b.v, a.d + b.d}; }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator-(Dual<T> a, Dual<T> b) { return {a.v - b.v, a.d - b.d}; }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator-(Dual<T> a) { return {-a.v, -a.d}; }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator*(Dual<T> a, Dual<T> b) { return {a.v * b.v, a.v * b.d + a.d * b.v}; }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator*(T a, Dual<T> b) { return {a * b.v, a * b.d}; }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator*(Dual<T> a, T b) { return {a.v * b, a.d * b}; }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator+(Dual<T> a, T b) { return {a.v + b, a.d}; }
template <class T> __host__ __device__ __forceinline__ Dual<T> operator/(Dual<T> a, Dual<T> b) {
  T q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}

// value / sincos for plain and dual scalars
__host__ __device__ __forceinline__ double val(double a) { return a; }
__host__ __device__ __forceinline__ float val(float a) { return a; }
template <class T> __host__ __device__ __forceinline__ T val(Dual<T> a) { return a.v; }

#ifdef __CUDACC__
// One out-of-line copy of each trigonometric routine per translation unit: the
// RK4 routines call them twelve times per step in several scalar types, and
// inlining every call site multiplies the code the instruction cache must hold
// (the iteration kernels run 24 warps per SM at different points of the code).
static __device__ __noinline__ void sincos_out(double a, double* s, double* c) { sincos(a, s, c); }
static __device__ __noinline__ void sincosf_out(float a, float* s, float* c) { sincosf(a, s, c); }
#endif
__host__ __device__ __forceinline__ void sincos_s(double a, double* s, double* c) {
#ifdef __CUDA_ARCH__
  sincos_out(a, s, c);
#else
  *s = ::sin(a);
  *c = ::cos(a);
#endif
}
__host__ __device__ __forceinline__ void sincos_s(float a, float* s, float* c) {
#ifdef __CUDA_ARCH__
  sincosf_out(a, s, c);
#else
  *s = ::sinf(a);
  *c = ::cosf(a);
#endif
}
template <class T>
__host__ __device__ __forceinline__ void sincos_s(Dual<T> a, Dual<T>* s, Dual<T>* c) {
  T sv, cv;
  sincos_s(a.v, &sv, &cv);
  *s = Dual<T>{sv, cv * a.d};
  *c = Dual<T>{cv, -sv * a.d};
}

template <class S> struct Base { typedef S type; };
template <class T> struct Base<Dual<T>> { typedef T type; };

// constant of scalar type S (a Dual constant has a zero derivative)
template <class S>
struct CstOf {
  static __host__ __device__ __forceinline__ S make(S v) { return v; }
};
template <class T>
struct CstOf<Dual<T>> {
  static __host__ __device__ __forceinline__ Dual<T> make(T v) { return Dual<T>{v, T(0)}; }
};
template <class S>
__host__ __device__ __forceinline__ S cst(typename Base<S>::type v) {
  return CstOf<S>::make(v);
}

// ------------------------------------------------------------ model constants
// Rigid-body quadrotor with four rotor thrusts ("+" layout), Sec. VI model
// family; constants fixed by the design readings.
constexpr double kMass = 0.5;
constexpr double kGrav = 9.81;
constexpr double kJx = 2.32e-3, kJy = 2.32e-3, kJz = 4.00e-3;
constexpr double kArm = 0.175;
constexpr double kYaw = 0.01;
constexpr double kHover = kMass * kGrav / 4.0;
constexpr double kUmax = 2.0 * kHover;
// tracking weights (diagonal), terminal weight factor
__host__ __device__ __forceinline__ double q_weight(int j) {  // j = component 0..11 of one quad
  return j < 3 ? 10.0 : (j < 9 ? 1.0 : 0.1);
}
constexpr double kRweight = 0.1;
constexpr double kQNscale = 10.0;

}  // namespace bipm
