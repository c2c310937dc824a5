// Complex element type of the CUDA-core kernels (paper Sec. 2: the operation is
// defined over the complex field; Sec. 3: T in {single, double} x {real,
// complex}).  Storage is interleaved (real part, imaginary part), the layout of
// C99 complex types, std::complex and cuComplex.
#pragma once

#include <cuda_runtime.h>

namespace kron {

template <typename R>
struct __align__(2 * sizeof(R)) cplx {
    R re, im;
    cplx() = default;
    __host__ __device__ constexpr cplx(R r, R i = R(0)) : re(r), im(i) {}
};
typedef cplx<float> cf32;
typedef cplx<double> cf64;

template <typename T> struct is_cplx { static constexpr bool value = false; };
template <typename R> struct is_cplx<cplx<R>> { static constexpr bool value = true; };

template <typename R>
__host__ __device__ __forceinline__ cplx<R> operator*(cplx<R> a, cplx<R> b) {
    return cplx<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R>
__host__ __device__ __forceinline__ cplx<R> operator+(cplx<R> a, cplx<R> b) {
    return cplx<R>(a.re + b.re, a.im + b.im);
}

// a * b + c: four real fused multiply-adds.
__device__ __forceinline__ cf32 madd(cf32 a, cf32 b, cf32 c) {
    return cf32(__fmaf_rn(a.re, b.re, __fmaf_rn(-a.im, b.im, c.re)), __fmaf_rn(a.re, b.im, __fmaf_rn(a.im, b.re, c.im)));
}
__device__ __forceinline__ cf64 madd(cf64 a, cf64 b, cf64 c) {
    return cf64(__fma_rn(a.re, b.re, __fma_rn(-a.im, b.im, c.re)), __fma_rn(a.re, b.im, __fma_rn(a.im, b.re, c.im)));
}
__device__ __forceinline__ float madd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double madd(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename R>
__device__ __forceinline__ cplx<R> conj_of(cplx<R> v) { return cplx<R>(v.re, -v.im); }

}  // namespace kron
