// Two-cells-per-thread stream-and-collide for 16-bit storage (FP16 and BF16
// deviations), periodic lattices with an even nx: two-lattice pull streaming
// and both steps of the in-place AA pattern.
//
// The per-cell kernel spends most of its issue slots on work that does not
// scale with the bytes it moves: 16-bit loads and stores, one conversion per
// population and per-cell address arithmetic. Here a thread owns the cell
// pair (x0, x0 + 1), x0 even, and shares the y/z neighbour arithmetic between
// them:
//  * c_x = 0: the pair's two populations are one aligned 32-bit word of the
//    pull source row;
//  * c_x = +-1: either two aligned words (the pair's word and its left or
//    right neighbour, merged with one byte permute; LD_WORDS) or two 16-bit
//    loads (LD_HALVES); L1 serves the overlap between neighbouring threads;
//  * stores: one 32-bit word per direction, packed by a single paired
//    conversion.
// The collision is the same function as the per-cell kernel, evaluated on
// both cells at once with the paired FP32 instructions (lane type F2 of
// lattice.cuh), so both kernels produce bit-identical states. A first version that passed the
// x-shifted halves between lanes with shuffles (so that every load was one
// aligned word) ran slower than the per-cell kernel: the extra loads of the
// first and last lane of each row segment and the shuffle latency cost more
// than the L1 traffic they saved. Register caps matter more than the load
// scheme: at 64 registers (4 blocks of 256 per SM) the force-along-x form
// reaches ~0.86 of the measured copy bandwidth, at 96 registers ~0.67.
#pragma once

#include "k_step.cuh"

namespace hlbm {

template <class S>
struct Pair16;
template <>
struct Pair16<StoreF16> {
    __device__ static float2 unpack(unsigned w) {
        __half2 h;
        memcpy(&h, &w, 4);
        return __half22float2(h);
    }
    __device__ static unsigned pack(float lo, float hi) {
        const __half2 h = __floats2half2_rn(lo, hi);
        unsigned w;
        memcpy(&w, &h, 4);
        return w;
    }
};
template <>
struct Pair16<StoreBF16> {
    __device__ static float2 unpack(unsigned w) {
        return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
    }
    __device__ static unsigned pack(float lo, float hi) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        unsigned w;
        memcpy(&w, &h, 4);
        return w;
    }
};

// Block width in threads (cell pairs) along x: 64 when it divides the row's
// pair count, else 32, else the width (up to 128) that leaves the fewest idle
// threads; short rows take the next power of two.
inline int pair_block_x(int nx) {
    const int pairs = nx / 2;
    if (pairs <= 32) {
        int b = 1;
        while (b < pairs) b <<= 1;
        return b;
    }
    if (pairs % 64 == 0) return 64;
    if (pairs % 32 == 0) return 32;
    int best = 64, waste_best = 1 << 30;
    for (int b : {64, 32, 128, 96}) {
        const int waste = ((pairs + b - 1) / b) * b - pairs;
        if (waste < waste_best) {
            best = b;
            waste_best = waste;
        }
    }
    return best;
}

enum PairLoad { LD_WORDS = 0, LD_HALVES = 1 };

// The 2 x Q populations the pair (x0, x0 + 1) consumes, as float pairs
// (d0: cell x0, d1: cell x0 + 1). row_i = plane i at the pull source row of
// the pair's word (x0, y - c_y, z - c_z); xm1 / xp2 = offsets of x0 - 1 and
// x0 + 2 within that row (periodic).
template <int Q, class S, int LD>
__device__ __forceinline__ void pair_gather(const Planes<const typename S::T, Q>& fin, int cell, const Nbr<int>& nb,
                                            int xm1, int xp2, float* d0, float* d1) {
    using L = Lat<Q>;
    using P = Pair16<S>;
    using T = typename S::T;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        int o = 0;  // y/z part of the pull offset
        if (L::cy(i) > 0) o += nb.oym;
        if (L::cy(i) < 0) o += nb.oyp;
        if (L::cz(i) > 0) o += nb.ozm;
        if (L::cz(i) < 0) o += nb.ozp;
        const T* row = fin.p[i] + (cell + o);
        if (L::cx(i) == 0) {
            const float2 f2 = P::unpack(__ldg(reinterpret_cast<const unsigned*>(row)));
            d0[i] = f2.x;
            d1[i] = f2.y;
        } else if (LD == LD_WORDS) {
            // the word holding x0 - 1 starts at x0 - 2 (xm1 - 1); the one holding x0 + 2 at xp2
            const unsigned b = __ldg(reinterpret_cast<const unsigned*>(row));
            const unsigned w = L::cx(i) > 0
                                   ? __byte_perm(__ldg(reinterpret_cast<const unsigned*>(row + (xm1 - 1))), b, 0x5432)
                                   : __byte_perm(b, __ldg(reinterpret_cast<const unsigned*>(row + xp2)), 0x5432);
            const float2 f2 = P::unpack(w);
            d0[i] = f2.x;
            d1[i] = f2.y;
        } else if (L::cx(i) > 0) {  // sources x0 - 1, x0
            d0[i] = S::load_raw(row + xm1, 0);
            d1[i] = S::load_raw(row, 0);
        } else {  // sources x0 + 1, x0 + 2
            d0[i] = S::load_raw(row + 1, 0);
            d1[i] = S::load_raw(row + xp2, 0);
        }
    }
}

// The same gather keeping each direction's pair as one 32-bit word (lane 0 in
// the low half): 19 registers instead of 38, unpacked exactly where used.
// INPLACE (the odd AA step, whose source is also its destination): plain
// coherent loads instead of the read-only path, and only 16-bit loads on the
// x-shifted directions, so that a thread reads no population another thread
// of the launch writes.
template <class V, bool INPLACE, class P>
__device__ __forceinline__ V ld_pop(const P* p) {
    if constexpr (INPLACE) return *reinterpret_cast<const V*>(p);  // may alias this launch's stores
    else return __ldg(reinterpret_cast<const V*>(p));
}

template <int Q, class S, int LD, bool INPLACE = false>
__device__ __forceinline__ void pair_gather_words(const Planes<const typename S::T, Q>& fin, int cell,
                                                  const Nbr<int>& nb, int xm1, int xp2, unsigned* w) {
    using L = Lat<Q>;
    using T = typename S::T;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        int o = 0;  // y/z part of the pull offset
        if (L::cy(i) > 0) o += nb.oym;
        if (L::cy(i) < 0) o += nb.oyp;
        if (L::cz(i) > 0) o += nb.ozm;
        if (L::cz(i) < 0) o += nb.ozp;
        const T* row = fin.p[i] + (cell + o);
        if (L::cx(i) == 0) {
            w[i] = ld_pop<unsigned, INPLACE>(row);
        } else if (LD == LD_WORDS && !INPLACE) {
            const unsigned b = __ldg(reinterpret_cast<const unsigned*>(row));
            w[i] = L::cx(i) > 0 ? __byte_perm(__ldg(reinterpret_cast<const unsigned*>(row + (xm1 - 1))), b, 0x5432)
                                : __byte_perm(b, __ldg(reinterpret_cast<const unsigned*>(row + xp2)), 0x5432);
        } else {
            const unsigned lo = L::cx(i) > 0 ? ld_pop<unsigned short, INPLACE>(row + xm1)
                                             : ld_pop<unsigned short, INPLACE>(row + 1);  // sources x0 -+ 1
            const unsigned hi = L::cx(i) > 0 ? ld_pop<unsigned short, INPLACE>(row)
                                             : ld_pop<unsigned short, INPLACE>(row + xp2);  // sources x0, x0 + 2
            w[i] = lo | (hi << 16);
        }
    }
}

// Exact unpack of a 16-bit pair word to two FP32 lanes, as an instruction
// sequence the compiler does not merge between uses: a population is read
// twice (moments, then relaxation), and unpacking it again is cheaper than
// keeping both FP32 values live across the collision.
template <class S>
__device__ __forceinline__ F2 unpack_each_use(unsigned w);
template <>
__device__ __forceinline__ F2 unpack_each_use<StoreF16>(unsigned w) {
    F2 r;
    asm volatile(
        "{\n\t.reg .b16 l16, h16;\n\t.reg .f32 lo, hi;\n\tmov.b32 {l16, h16}, %1;\n\t"
        "cvt.f32.f16 lo, l16;\n\tcvt.f32.f16 hi, h16;\n\tmov.b64 %0, {lo, hi};\n\t}"
        : "=l"(r.v) : "r"(w));
    return r;
}
template <>
__device__ __forceinline__ F2 unpack_each_use<StoreBF16>(unsigned w) {
    F2 r;
    asm volatile(
        "{\n\t.reg .b32 lo, hi;\n\tshl.b32 lo, %1, 16;\n\tand.b32 hi, %1, 0xffff0000;\n\t"
        "mov.b64 %0, {lo, hi};\n\t}"
        : "=l"(r.v) : "r"(w));
    return r;
}

// Populations of a cell pair held as the loaded 32-bit words (lane 0 in the
// low half); d[i] unpacks direction i to the two FP32 lanes on each use.
template <class S, int Q>
struct PackedPairs {
    unsigned w[Q];
    __device__ __forceinline__ F2 operator[](int i) const { return unpack_each_use<S>(w[i]); }
};

#ifndef HLBM_PAIR_FX_BLOCKS
#define HLBM_PAIR_FX_BLOCKS 4
#endif
template <int FORM>
struct PairTraits {
    // the force-along-x form fits 64 registers (4 blocks per SM) with word loads; the
    // others take 80 (3 blocks) with 16-bit loads on the x-shifted directions
    static constexpr int kMinBlocks = FORM == FORM_SHIFT_FX ? HLBM_PAIR_FX_BLOCKS : 3;
    static constexpr int kLoad = FORM == FORM_SHIFT_FX ? LD_WORDS : LD_HALVES;
};

// MODE: MODE_TWO_LATTICE (pull from fin, store into fout at the cell pair),
// MODE_AA_EVEN (in place; read the pair's own slots i, write f*_i into the
// pair's own slot opp(i): the launcher passes fout with the planes permuted,
// so the store is the two-lattice one) or MODE_AA_ODD (in place; read slot
// opp(i) at x - c_i: fin with permuted planes and the pull gather; write slot i
// at x + c_i). In the AA steps every population is read and written by the
// same thread, so the in-place update needs no synchronisation.
// Block size and register budget of a paired kernel. The BF16 two-lattice
// force-along-x kernel runs at 56 registers in 128-thread blocks (9 blocks, 36
// resident warps per SM; measured at 384^3: 0.973 vs 0.955 of the copy
// bandwidth at 64 registers). The FP16 kernel (whose unpack costs more
// registers) and the in-place steps measured slower at 56 (FP16 0.919 vs 0.922,
// AA 0.855 / 0.892 vs 0.884 / 0.912), so they keep 256-thread blocks and the
// budget of PairTraits.
template <class S, int FORM, int MODE>
struct PairLaunch {
    static constexpr bool k56 = S::kind == 3 /* BF16 */ && FORM == FORM_SHIFT_FX && MODE == MODE_TWO_LATTICE;
    static constexpr int kThreads = k56 ? 128 : 256;
    static constexpr int kMinBlocks = k56 ? 9 : PairTraits<FORM>::kMinBlocks;
};

template <int Q, class S, int FORM, int MODE>
__global__ void __launch_bounds__(PairLaunch<S, FORM, MODE>::kThreads, PairLaunch<S, FORM, MODE>::kMinBlocks)
k_step_pair(Planes<const typename S::T, Q> fin, Planes<typename S::T, Q> fout, const float* __restrict__ varpi,
            Geometry g, Phys<float> ph, float s, float inv_s, const float* __restrict__ varpi3) {
    using P = Pair16<S>;
    using L = Lat<Q>;
    using T = typename S::T;
    const int xp = blockIdx.x * blockDim.x + threadIdx.x;  // pair index along x
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (2 * xp >= g.nx || y >= g.ny) return;
    const int x0 = 2 * xp;
    const int cell = x0 + g.nx * (y + g.ny * z);
    const Nbr<int> nb(g, x0, y, z);
    const int xm1 = x0 == 0 ? g.nx - 1 : -1;
    const int xp2 = x0 + 2 >= g.nx ? -x0 : 2;

    PackedPairs<S, Q> d;  // the loaded words; lane 0: cell x0, lane 1: cell x0 + 1
    if constexpr (MODE == MODE_AA_EVEN) {
#pragma unroll
        for (int i = 0; i < Q; ++i) d.w[i] = ld_pop<unsigned, true>(fin.p[i] + cell);
    } else if constexpr (MODE == MODE_AA_ODD) {
        pair_gather_words<Q, S, LD_HALVES, true>(fin, cell, nb, xm1, xp2, d.w);
    } else {
        pair_gather_words<Q, S, PairTraits<FORM>::kLoad>(fin, cell, nb, xm1, xp2, d.w);
    }

    // each post-collision pair of values is stored as soon as it is final: one 32-bit word at
    // the pair, or (odd AA step) at the pair shifted by c_i, split into two 16-bit stores when
    // the shift is along x
    const auto store = [&](int i, F2 v) {
        const float2 f = v.split();
        if constexpr (MODE == MODE_AA_ODD) {
            int o = 0;  // y/z part of the push offset
            if (L::cy(i) > 0) o += nb.oyp;
            if (L::cy(i) < 0) o += nb.oym;
            if (L::cz(i) > 0) o += nb.ozp;
            if (L::cz(i) < 0) o += nb.ozm;
            T* row = fout.p[i] + (cell + o);
            if (L::cx(i) == 0) {
                *reinterpret_cast<unsigned*>(row) = P::pack(f.x, f.y);
            } else if (L::cx(i) > 0) {  // targets x0 + 1, x0 + 2
                S::store_raw(row, 1, f.x);
                S::store_raw(row, xp2, f.y);
            } else {  // targets x0 - 1, x0
                S::store_raw(row, xm1, f.x);
                S::store_raw(row, 0, f.y);
            }
        } else {
            *reinterpret_cast<unsigned*>(fout.p[i] + cell) = P::pack(f.x, f.y);
        }
    };
    if (FORM == FORM_ANISO) {
        float2 v3[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) v3[a] = __ldg(reinterpret_cast<const float2*>(varpi3 + (size_t)a * g.N + cell));
        collide_aniso<Q, F2, S::scaled>(d, F2(v3[0].x, v3[0].y), F2(v3[1].x, v3[1].y), F2(v3[2].x, v3[2].y), ph, s,
                                        inv_s, store);
    } else {
        const float2 vp = __ldg(reinterpret_cast<const float2*>(varpi + cell));
        if (FORM == FORM_DRAG) collide_drag<Q, F2, S::scaled>(d, F2(vp.x, vp.y), ph, s, inv_s, store);
        else collide<Q, F2, S::scaled, FORM == FORM_SHIFT_FX>(d, F2(vp.x, vp.y), ph, s, inv_s, store);
    }
}

// Launch of the paired kernel; the caller has checked pair_applies(). The AA
// steps run in place (fin and fout are the same buffer) with the planes of
// their gathered (odd step) or stored (even step) side permuted to opp(i).
template <int Q, class S, int FORM, int MODE>
cudaError_t step_pair_impl(const LaunchCtx& c, const void* fin, void* fout, const float* varpi) {
    using T = typename S::T;
    Geometry g{c.nx, c.ny, c.nz, 0, 0, 0, (size_t)c.nx * c.ny * c.nz};
    const Phys<float> ph = make_phys<float, Q>(c.tau, c.F);
    constexpr int threads = PairLaunch<S, FORM, MODE>::kThreads;
    const int bx = pair_block_x(c.nx);
    const int by = bx >= threads ? 1 : threads / bx;
    const dim3 blk(bx, by, 1);
    const dim3 grd((c.nx / 2 + bx - 1) / bx, (c.ny + by - 1) / by, c.nz);
    Planes<const T, Q> a;
    Planes<T, Q> b;
    for (int i = 0; i < Q; ++i) {
        const int ia = MODE == MODE_AA_ODD ? opp<Q>(i) : i;
        const int ib = MODE == MODE_AA_EVEN ? opp<Q>(i) : i;
        a.p[i] = static_cast<const T*>(fin) + (size_t)ia * g.N;
        b.p[i] = static_cast<T*>(fout) + (size_t)ib * g.N;
    }
    k_step_pair<Q, S, FORM, MODE><<<grd, blk, 0, c.stream>>>(a, b, varpi, g, ph, float(c.scale),
                                                             float(1.0 / c.scale), c.varpi3);
    return cudaGetLastError();
}

// The paired kernel covers periodic lattices with an even nx (aligned pair
// words in every plane) and 32-bit indices: two-lattice steps in every
// collision form, AA steps in the equilibrium-shift forms.
inline bool pair_applies(const LaunchCtx& c, int mode) {
    if (c.variant != 0 || c.wall[0] || c.wall[1] || c.wall[2] || c.links || c.nx < 2 || (c.nx % 2) != 0 ||
        (size_t)c.q * c.nx * c.ny * c.nz >= ((size_t)1 << 31))
        return false;
    if (mode == MODE_TWO_LATTICE) return true;
    const int form = step_form(c, c.q);
    return (mode == MODE_AA_EVEN || mode == MODE_AA_ODD) && (form == FORM_SHIFT_FX || form == FORM_SHIFT);
}

template <int Q, class S, int MODE>
cudaError_t step_pair_forms(const LaunchCtx& c, const void* fin, void* fout, const float* varpi) {
    if constexpr (MODE == MODE_TWO_LATTICE) {
        switch (step_form(c, Q)) {
            case FORM_SHIFT_FX: return step_pair_impl<Q, S, FORM_SHIFT_FX, MODE>(c, fin, fout, varpi);
            case FORM_SHIFT: return step_pair_impl<Q, S, FORM_SHIFT, MODE>(c, fin, fout, varpi);
            case FORM_DRAG: return step_pair_impl<Q, S, FORM_DRAG, MODE>(c, fin, fout, varpi);
            default: return step_pair_impl<Q, S, FORM_ANISO, MODE>(c, fin, fout, varpi);
        }
    } else {
        return step_form(c, Q) == FORM_SHIFT_FX ? step_pair_impl<Q, S, FORM_SHIFT_FX, MODE>(c, fin, fout, varpi)
                                                : step_pair_impl<Q, S, FORM_SHIFT, MODE>(c, fin, fout, varpi);
    }
}

template <int Q, class S>
cudaError_t step_pair_modes(const LaunchCtx& c, int mode, const void* fin, void* fout, const float* varpi) {
    switch (mode) {
        case MODE_TWO_LATTICE: return step_pair_forms<Q, S, MODE_TWO_LATTICE>(c, fin, fout, varpi);
        case MODE_AA_EVEN: return step_pair_forms<Q, S, MODE_AA_EVEN>(c, fin, fout, varpi);
        case MODE_AA_ODD: return step_pair_forms<Q, S, MODE_AA_ODD>(c, fin, fout, varpi);
    }
    return cudaErrorInvalidValue;
}

// Step kernels of a 16-bit storage policy: the paired kernel where it
// applies, else the per-cell kernels.
template <class S>
cudaError_t step_for_storage16(const LaunchCtx& c, int mode, const void* fin, void* fout, const float* varpi) {
    if (pair_applies(c, mode)) {
        if (c.q == 9) return step_pair_modes<9, S>(c, mode, fin, fout, varpi);
        if (c.q == 19) return step_pair_modes<19, S>(c, mode, fin, fout, varpi);
        return cudaErrorInvalidValue;
    }
    return step_for_storage<S>(c, mode, fin, fout, varpi);
}

}  // namespace hlbm
