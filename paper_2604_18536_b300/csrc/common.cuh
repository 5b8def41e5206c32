// Shared device-side definitions of libins: complex arithmetic, the geometry
// record every stencil kernel receives, and index helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ins {

template <typename T>
struct alignas(2 * sizeof(T)) cplx {
    T re, im;
};

template <typename T>
__device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T>
__device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T>
__device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
    return {fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}
template <typename T>
__device__ __forceinline__ cplx<T> cconj(cplx<T> a) { return {a.re, -a.im}; }
template <typename T>
__device__ __forceinline__ cplx<T> cscale(cplx<T> a, T s) { return {a.re * s, a.im * s}; }
// read-only cached load of a complex value
__device__ __forceinline__ cplx<double> ldg_c(const cplx<double>* p) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    return {v.x, v.y};
}
__device__ __forceinline__ cplx<float> ldg_c(const cplx<float>* p) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return {v.x, v.y};
}
// multiply by -i
template <typename T>
__device__ __forceinline__ cplx<T> cmul_mi(cplx<T> a) { return {a.im, -a.re}; }

// Per-direction stencil coefficients, all in the field type T, each an array
// over the cell index of that direction (length n_a). d = cell widths,
// h = centre-to-centre distances (h[i] between cells i and i+1).
enum Coef {
    C_INV_H = 0,     // 1/h[i]
    C_INV_D,         // 1/d[i]
    C_CONV_AA,       // 0.25/h[i]   (self term: ((u_i+u_{i+1})^2 - (u_{i-1}+u_i)^2) * 0.25/h)
    C_CONV_AB,       // 0.5/d[i]    (cross term along this direction as the flux direction)
    C_WL,            // d[i]/(d[i]+d[i+1])  volume weight of the left value
    C_WR,            // d[i+1]/(d[i]+d[i+1])
    C_DIFF_AP,       // nu/(d[i+1] h[i])  same-direction diffusion, upper neighbour
    C_DIFF_AM,       // nu/(d[i] h[i])    same-direction diffusion, lower neighbour
    C_DIFF_BP,       // nu/(h[i] d[i])    cross-direction diffusion, upper neighbour
    C_DIFF_BM,       // nu/(h[i-1] d[i])  cross-direction diffusion, lower neighbour
    C_COUNT
};

// read-only loads of coefficient tables (a double-float overload sits with that type)
__device__ __forceinline__ float geo_ldg(const float* p) { return __ldg(p); }
__device__ __forceinline__ double geo_ldg(const double* p) { return __ldg(p); }

template <typename T>
struct Geo {
    int nx, ny, nz;          // nz = 1 in 2-D
    int wall_y;              // 1: y is a no-slip wall direction, x and z periodic
    const T* c[3];           // c[a] -> C_COUNT arrays of n_a values, array m at c[a] + m*n_a
    T fx, fy, fz;            // body force
    __device__ __forceinline__ T coef(int a, int m, int i) const {
        int n = a == 0 ? nx : (a == 1 ? ny : nz);
        return geo_ldg(c[a] + (size_t)m * n + i);
    }
};

__device__ __forceinline__ int wrap(int i, int n) {
    // i in [-n, 2n)
    return i < 0 ? i + n : (i >= n ? i - n : i);
}

}  // namespace ins
