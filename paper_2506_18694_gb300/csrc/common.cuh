// Shared device helpers: complex arithmetic on interleaved float2/double2 and the
// per-node one-dimensional Q1 weights from which every operator is built.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hh {

// Programmatic dependent launch: let the next kernel in the stream start launching now,
// then wait until every kernel this one depends on has finished and flushed its writes.
// Every kernel calls this before its first global memory access.
__device__ __forceinline__ void pdl_entry() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename T> struct VecOf;
template <> struct VecOf<float> { using type = float2; };
template <> struct VecOf<double> { using type = double2; };
template <typename T> using vec2 = typename VecOf<T>::type;

// Complex value held in registers.
template <typename T> struct Cx {
    T re, im;
};

template <typename T> __host__ __device__ __forceinline__ Cx<T> cx(T r, T i) { return Cx<T>{r, i}; }
template <typename T> __device__ __forceinline__ Cx<T> ld(const vec2<T>* p, long long i) {
    vec2<T> v = p[i];
    return Cx<T>{v.x, v.y};
}
template <typename T> __device__ __forceinline__ void st(vec2<T>* p, long long i, Cx<T> v) {
    vec2<T> w;
    w.x = v.re;
    w.y = v.im;
    p[i] = w;
}
template <typename T> __device__ __forceinline__ Cx<T> operator+(Cx<T> a, Cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T> __device__ __forceinline__ Cx<T> operator-(Cx<T> a, Cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T> __device__ __forceinline__ Cx<T> operator*(T s, Cx<T> a) { return {s * a.re, s * a.im}; }
// Complex product with the fused multiply-adds written out, so that the rounding does not
// depend on how the compiler contracts the expression in a given kernel.
template <typename T> __device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b) {
    return {fma(a.re, b.re, -(a.im * b.im)), fma(a.re, b.im, a.im * b.re)};
}
// a + s * b with real s
template <typename T> __device__ __forceinline__ Cx<T> fma_r(T s, Cx<T> b, Cx<T> a) {
    return {fma(s, b.re, a.re), fma(s, b.im, a.im)};
}
// a + c * b with complex c
template <typename T> __device__ __forceinline__ Cx<T> fma_c(Cx<T> c, Cx<T> b, Cx<T> a) {
    return {fma(c.re, b.re, fma(-c.im, b.im, a.re)), fma(c.re, b.im, fma(c.im, b.re, a.im))};
}
// a / 2 rounded on its own.  The intrinsics are never fused into a following add, so every kernel
// rounds the interpolation and restriction halves the same way: for subnormal values a / 2 is
// inexact, and a contraction of "x + a / 2" into one fused multiply-add in some kernels but not in
// others would change the last bit.
__device__ __forceinline__ float half_rn1(float a) { return __fmul_rn(0.5f, a); }
__device__ __forceinline__ double half_rn1(double a) { return __dmul_rn(0.5, a); }
template <typename T> __device__ __forceinline__ Cx<T> half_rn(Cx<T> a) { return {half_rn1(a.re), half_rn1(a.im)}; }
template <typename T> __device__ __forceinline__ Cx<T> cinv(Cx<T> a) {
    T d = fma(a.re, a.re, a.im * a.im);
    T s = T(1) / d;
    return {a.re * s, -a.im * s};
}

// Grid of one level: nodes 0..n per axis, x fastest.  dir[s] = 1 if side s
// (-x,+x,-y,+y,-z,+z) carries the Dirichlet condition, 0 for Sommerfeld.
struct GridDesc {
    int dim;
    int n;
    int nn;
    long long N;
    double h;
    int dir[6];
};

// Coefficient triple of an operator c_K K + c_M M + c_G M_Gamma (c_K is real for
// every operator the solver uses).
template <typename T> struct OpCoef {
    T cK;
    Cx<T> cM;
    Cx<T> cG;
};

// One-dimensional Q1 weights of the node with coordinate i along one axis:
// stiffness (1/h)[-1 2 -1] and mass (h/6)[1 4 1], halved at the two ends, with the
// weight of a neighbour that is a Dirichlet node (an eliminated unknown) set to 0.
template <typename T> struct Row1 {
    T kl, kc, kr;   // stiffness weights of neighbours i-1, i, i+1
    T ml, mc, mr;   // mass weights
    int lo, hi;     // clamped neighbour coordinates (always inside 0..n)
    bool masked;    // node itself is Dirichlet
    bool face;      // node lies on a Sommerfeld side of this axis
};

template <typename T>
__device__ __forceinline__ Row1<T> row1(int i, int n, int dlo, int dhi, T h, T ih) {
    Row1<T> r;
    const bool has_l = i > 0, has_r = i < n;
    const bool nl = has_l && !(i - 1 == 0 && dlo);
    const bool nr = has_r && !(i + 1 == n && dhi);
    const T cnt = T(has_l) + T(has_r);
    r.kc = cnt * ih;
    r.mc = cnt * h * T(1.0 / 3.0);
    r.kl = nl ? -ih : T(0);
    r.kr = nr ? -ih : T(0);
    r.ml = nl ? h * T(1.0 / 6.0) : T(0);
    r.mr = nr ? h * T(1.0 / 6.0) : T(0);
    r.lo = has_l ? i - 1 : i;
    r.hi = has_r ? i + 1 : i;
    r.masked = (i == 0 && dlo) || (i == n && dhi);
    r.face = (i == 0 && !dlo) || (i == n && !dhi);
    return r;
}

}  // namespace hh
