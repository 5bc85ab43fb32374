// Deterministic per-block fold of the FP64 diagnostics (mass, momentum, plane
// flux, residual, max speed), shared by the single-lattice and the batched
// reduction kernels.
//
// GB300 runs FP64 arithmetic (and float<->double conversion) at a small
// fraction of its FP32 rate, so the fold keeps FP64 work to what the sums
// need:
//  * each thread converts its cell's drho and j to double (4 conversions);
//    the F/2 shift of rho*u is added once per block from the count of fluid
//    cells instead of once per cell (shift form only);
//  * the residual max|du| and the speed max|u| stay in the arithmetic type:
//    a max is exact in any precision and order-independent, and is folded on
//    the bit patterns (non-negative values order like unsigned integers), so
//    a NaN anywhere reaches the result instead of being dropped by fmax;
//  * the five sums are folded through shared memory in a fixed order (40
//    threads sum interleaved segments, 5 threads combine them), not with
//    shuffle trees: the result does not depend on scheduling.
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

// One thread's diagnostics over its cells (one or two). s[0] = sum drho,
// s[1..3] = sum j (plus F/2 and the drag factor when `shifted` is set), s[4]
// = the part of s[1] on the x = nx-1 plane; fluid / plane count the cells
// behind s[1..3] / s[4].
template <class C>
struct DiagCell {
    double s[5] = {0, 0, 0, 0, 0};
    C du = C(0), um = C(0);
    int fluid = 0, plane = 0;
    bool shifted = false;  // F/2 already inside s[1..4]
};

constexpr int kDiagPad = 264;  // row stride of the fold buffer (conflict-free 64-bit reads)

struct DiagShared {
    double sum[5][kDiagPad];
    double seg[5][8];
    unsigned long long mx[2];
};

// Fold the block's cells into out[8] (drho sum, rho*u sum (3), plane flux, 0,
// max|du|, max|u|). Every thread of the block calls it; nt = threads (a
// multiple of 8, at most 256), F = the force in double, MAXC = the most
// cells a thread holds.
template <class C, int MAXC = 1>
__device__ __forceinline__ void diag_fold(const DiagCell<C>& a, DiagShared& sh, int t, int nt, double Fx, double Fy,
                                          double Fz, double* out) {
    using B = DiagBits<C>;
    if (t < 2) sh.mx[t] = 0ull;
#pragma unroll
    for (int k = 0; k < 5; ++k) sh.sum[k][t] = a.s[k];
    __syncthreads();
    const typename B::U bdu = B::warp_max(B::bits(a.du));
    const typename B::U bum = B::warp_max(B::bits(a.um));
    if ((t & 31) == 0) {
        atomicMax(reinterpret_cast<typename B::U*>(&sh.mx[0]), bdu);
        atomicMax(reinterpret_cast<typename B::U*>(&sh.mx[1]), bum);
    }
    // the counts are exact integers; the barriers also publish sum[] and mx[]
    int nfluid = 0, nplane = 0;
#pragma unroll
    for (int c = 1; c <= MAXC; ++c) {
        nfluid += __syncthreads_count(!a.shifted && a.fluid >= c);
        nplane += __syncthreads_count(!a.shifted && a.plane >= c);
    }
    if (t < 40) {
        const int k = t >> 3, sg = t & 7, per = nt >> 3;
        double v = sh.sum[k][sg];
        for (int m = 1; m < per; ++m) v += sh.sum[k][m * 8 + sg];
        sh.seg[k][sg] = v;
    }
    __syncthreads();
    if (t < 8) {
        double v = 0.0;
        if (t < 5) {
            v = sh.seg[t][0];
#pragma unroll
            for (int m = 1; m < 8; ++m) v += sh.seg[t][m];
            const double half = 0.5 * (t == 1 || t == 4 ? Fx : t == 2 ? Fy : t == 3 ? Fz : 0.0);
            if (t > 0) v += half * (double)(t == 4 ? nplane : nfluid);
        } else if (t >= 6) {
            v = B::value(*reinterpret_cast<const typename B::U*>(&sh.mx[t - 6]));
        }
        out[t] = v;
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
