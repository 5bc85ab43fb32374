// Deterministic per-block fold of the FP64 diagnostics (mass, momentum, plane
// flux, residual, max speed), shared by the single-lattice and the batched
// reduction kernels.
//
// GB300 runs FP64 arithmetic (and float<->double conversion) at a small
// fraction of its FP32 rate, and a fold built from long dependent chains of
// FP64 adds is latency-bound. So:
//  * a thread first adds its own few cells (at most four) in the arithmetic
//    type; the rounding of that short sum is far below the FP32 rounding of
//    each cell's own moments, and every sum beyond the thread is FP64;
//  * the F/2 shift of rho*u is added once per block from the exact count of
//    fluid cells instead of once per cell (shift form only);
//  * max|du| and max|u| stay in the arithmetic type: a max is exact in any
//    precision and order-free, and is folded on the bit patterns
//    (non-negative values order like unsigned integers), so a NaN anywhere
//    reaches the result instead of being dropped by fmax;
//  * the five sums are folded through shared memory by one warp per
//    quantity: each lane adds a fixed strided set, then a fixed shuffle tree
//    (dependency depth nt/32 - 1 + 5 instead of a 38-long chain). The result
//    does not depend on scheduling.
#pragma once
#include <cuda_runtime.h>

namespace hlbm {

template <class C>
struct DiagBits;
template <>
struct DiagBits<float> {
    using U = unsigned;
    __device__ static U bits(float v) { return __float_as_uint(v); }
    __device__ static double value(U b) { return (double)__uint_as_float(b); }
    __device__ static U warp_max(U b) { return __reduce_max_sync(0xffffffffu, b); }
};
template <>
struct DiagBits<double> {
    using U = unsigned long long;
    __device__ static U bits(double v) { return (U)__double_as_longlong(v); }
    __device__ static double value(U b) { return __longlong_as_double((long long)b); }
    __device__ static U warp_max(U b) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const U c = __shfl_xor_sync(0xffffffffu, b, o);
            b = c > b ? c : b;
        }
        return b;
    }
};

// max that keeps a NaN from either side
template <class C>
__device__ __forceinline__ C nan_max(C a, C b) {
    return (b > a || b != b) ? b : a;
}

// One thread's diagnostics over its cells. p[0] = sum drho, p[1..3] = sum j
// (plus F/2 and the drag factor when `shifted` is set), p[4] = the part of
// p[1] on the x = nx-1 plane, all in the arithmetic type; fluid / plane count
// the cells behind p[1..3] / p[4].
template <class C>
struct DiagCell {
    C p[5] = {C(0), C(0), C(0), C(0), C(0)};
    C du = C(0), um = C(0);
    int fluid = 0, plane = 0;
    bool shifted = false;  // F/2 already inside p[1..4]
};

struct DiagShared {
    double sum[5][256];
    unsigned long long mx[2];
    int cnt[2];
};

// Fold the block's cells into out[8] (drho sum, rho*u sum (3), plane flux, 0,
// max|du|, max|u|). Every thread of the block calls it; nt = threads (a
// multiple of 32, from 192 to 256), F = the force in double.
template <class C>
__device__ __forceinline__ void diag_fold(const DiagCell<C>& a, DiagShared& sh, int t, int nt, double Fx, double Fy,
                                          double Fz, double* out) {
    using B = DiagBits<C>;
    if (t < 2) {
        sh.mx[t] = 0ull;
        sh.cnt[t] = 0;
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) sh.sum[k][t] = (double)a.p[k];
    __syncthreads();
    const typename B::U bdu = B::warp_max(B::bits(a.du));
    const typename B::U bum = B::warp_max(B::bits(a.um));
    const int nf = __reduce_add_sync(0xffffffffu, a.shifted ? 0 : a.fluid);
    const int np = __reduce_add_sync(0xffffffffu, a.shifted ? 0 : a.plane);
    const int lane = t & 31, warp = t >> 5;
    if (lane == 0) {
        atomicMax(reinterpret_cast<typename B::U*>(&sh.mx[0]), bdu);
        atomicMax(reinterpret_cast<typename B::U*>(&sh.mx[1]), bum);
        atomicAdd(&sh.cnt[0], nf);  // integers: exact in any order
        atomicAdd(&sh.cnt[1], np);
    }
    __syncthreads();
    if (warp < 5) {
        const int k = warp;
        double v = sh.sum[k][lane];
        for (int m = 32 + lane; m < nt; m += 32) v += sh.sum[k][m];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) {
            const double half = 0.5 * (k == 1 || k == 4 ? Fx : k == 2 ? Fy : k == 3 ? Fz : 0.0);
            if (k > 0) v += half * (double)(k == 4 ? sh.cnt[1] : sh.cnt[0]);
            out[k] = v;
        }
    } else if (warp == 5 && lane == 0) {
        out[5] = 0.0;
        out[6] = B::value(*reinterpret_cast<const typename B::U*>(&sh.mx[0]));
        out[7] = B::value(*reinterpret_cast<const typename B::U*>(&sh.mx[1]));
    }
}

// Deterministic fold of one column of a partials array (stride 8 doubles):
// sums in FP64 in a fixed order, maxima on the bit patterns.
__device__ __forceinline__ double fold_column(const double* partials, size_t n, int col, double* buf /*[256]*/) {
    const int t = threadIdx.x;
    const bool is_max = col >= 6;
    double v = 0.0;
    unsigned long long b = 0ull;
    for (size_t i = t; i < n; i += blockDim.x) {
        const double p = partials[i * 8 + col];
        if (is_max) {
            const unsigned long long pb = (unsigned long long)__double_as_longlong(p);
            b = pb > b ? pb : b;
        } else {
            v += p;
        }
    }
    if (is_max) v = __longlong_as_double((long long)b);
    buf[t] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (t < s) {
            if (is_max) {
                const unsigned long long x = (unsigned long long)__double_as_longlong(buf[t]);
                const unsigned long long y = (unsigned long long)__double_as_longlong(buf[t + s]);
                buf[t] = __longlong_as_double((long long)(y > x ? y : x));
            } else {
                buf[t] += buf[t + s];
            }
        }
        __syncthreads();
    }
    return buf[0];
}

}  // namespace hlbm
