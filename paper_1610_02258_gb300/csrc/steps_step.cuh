// Device building blocks of the operator-split step (Parallel STEPS,
// Algorithm 1) and the per-tile step body shared by the plain and batched
// kernels. Included by one translation unit per kernel family; everything
// here has internal linkage.
//
// Compiled with -fmad=false: every floating-point operation that decides an
// integer (a reaction time, a reaction choice, a rounded trial count) is a
// single IEEE operation in the order written, so the same formulas evaluated
// on a host give the same bits.
#pragma once

#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>

#include "steps_internal.h"
#else
#include "steps_device.h"
#endif

namespace steps {
namespace {


// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two
// 32x32->64 multiplies with the Weyl key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1,
                                               uint32_t c2, uint32_t c3) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        c0 = n0;
        c1 = (uint32_t)p1;
        c2 = n2;
        c3 = (uint32_t)p0;
    }
    return make_uint4(c0, c1, c2, c3);
}

__device__ __forceinline__ uint32_t word_of(const uint4 &b, uint32_t k) {
    return k == 0 ? b.x : k == 1 ? b.y : k == 2 ? b.z : b.w;
}

// ---- TMA (bulk async copy) global -> shared, completed on an mbarrier
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Prefetch into L2; bytes: multiple of 16, address 16-byte aligned.
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// bytes: multiple of 16; both addresses 16-byte aligned
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// The waiting thread may be suspended for up to about 0.5 us per try (the
// hint) instead of spinning, leaving the issue slots to other warps.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(500u)
        : "memory");
    return ok != 0;
}

// Waits for the phase with the given parity to complete, for at most `limit`
// clock cycles (by default 2^30, ~0.5 s); returns false when the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit = 1ll << 30) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

// Natural log in single precision from the atanh series:
// x = 2^e f, f in (sqrt(1/2), sqrt(2)]; ln f = 2 atanh(s), s = (f-1)/(f+1),
// summed to s^11; e*ln2 added as a high part (exact for |e| < 2^8) and a low part.
__device__ __forceinline__ float steps_logf(float x) {
    const uint32_t u = __float_as_uint(x);
    int e = (int)((u >> 23) & 0xffu) - 127;
    float f = __uint_as_float((u & 0x007fffffu) | 0x3f800000u);
    if (f > 1.41421356f) {
        f = __fmul_rn(f, 0.5f);
        e = e + 1;
    }
    const float s = __fdiv_rn(__fsub_rn(f, 1.0f), __fadd_rn(f, 1.0f));
    const float z = __fmul_rn(s, s);
    float p = 0.0909090909f;
    p = __fadd_rn(__fmul_rn(p, z), 0.111111111f);
    p = __fadd_rn(__fmul_rn(p, z), 0.142857143f);
    p = __fadd_rn(__fmul_rn(p, z), 0.2f);
    p = __fadd_rn(__fmul_rn(p, z), 0.333333333f);
    p = __fadd_rn(__fmul_rn(p, z), 1.0f);
    const float lnf = __fmul_rn(__fadd_rn(s, s), p);
    const float fe = __int2float_rn(e);
    const float lo = __fadd_rn(__fmul_rn(fe, 1.42860682e-06f), lnf);
    return __fadd_rn(__fmul_rn(fe, 0.693145752f), lo);
}

// Uniform in (0, 1]: ((w >> 8) + 1) * 2^-24, exact in float.
__device__ __forceinline__ float unit24f(uint32_t w) {
    return __fmul_rn(__uint2float_rn((w >> 8) + 1u), 5.9604644775390625e-08f);
}

// Reaction table of a tile in shared memory, one broadcast load per reaction
// and field group. p[r] = (k, byte offset of row ia, byte offset of row ib,
// flags) with flags bits 0-7 = sub, bit 8 = c takes the factor 1/(N_A V),
// bit 9 = order 0; chg[r] = species (bytes 0-7) and deltas (bytes 8-15) of
// the nchg[r] species reaction r changes.
struct RxnTab {
    float4 p[kMaxReac];
    uint4 chg[kMaxReac];
    int32_t nchg[kMaxReac];
    uint32_t need[kMaxReac];
};

template <int BLOCK>
__device__ __forceinline__ void build_rxn_tab(const ModelDev &m, RxnTab &tb) {
    for (int r = threadIdx.x; r < m.R; r += BLOCK) {
        const ReacDesc &d = m.reac[r];
        const uint32_t fl = (uint32_t)d.sub | (d.type == kOrder2 || d.type == kDimer ? 0x100u : 0u) |
                            (d.type == kOrder0 ? 0x200u : 0u);
        tb.p[r] = make_float4(d.k, __uint_as_float((uint32_t)(d.ia * BLOCK * 4)),
                              __uint_as_float((uint32_t)(d.ib * BLOCK * 4)), __uint_as_float(fl));
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        for (int q = 0; q < d.nchg; ++q) {
            w[q >> 2] |= (uint32_t)(uint8_t)d.chg_s[q] << (8 * (q & 3));
            w[2 + (q >> 2)] |= (uint32_t)(uint8_t)d.chg_d[q] << (8 * (q & 3));
        }
        tb.chg[r] = make_uint4(w[0], w[1], w[2], w[3]);
        tb.nchg[r] = d.nchg;
        tb.need[r] = d.need;
    }
}

// Mass-action propensity in float, a = ((c x) y): order 0: c = k / (1/(N_A V)),
// x = y = 1; order 1: c = k, x = N, y = 1; order 2: c = k (1/(N_A V)),
// x = N_a, y = N_b; dimer: the same with y = N - 1. cnt points at the tet's
// column of the count tile (row S all ones); q is the reaction's table entry.
__device__ __forceinline__ float propensity(const float4 q, const int32_t *cnt, float inv_nav, bool has_order0) {
    const uint32_t fl = __float_as_uint(q.w);
    const int32_t x = *reinterpret_cast<const int32_t *>(reinterpret_cast<const char *>(cnt) + __float_as_uint(q.y));
    const int32_t y = *reinterpret_cast<const int32_t *>(reinterpret_cast<const char *>(cnt) + __float_as_uint(q.z)) -
                      (int32_t)(fl & 0xFFu);
    float c = __fmul_rn(q.x, (fl & 0x100u) ? inv_nav : 1.0f);
    if (has_order0 && (fl & 0x200u)) c = __fdiv_rn(q.x, inv_nav);
    return __fmul_rn(__fmul_rn(c, __int2float_rn(x)), __int2float_rn(y));
}

// Model access of the step body. RtModel reads a model given at run time
// (kernel parameters and the tile's reaction table). A model compiled into a
// kernel at run time (steps_spec.cpp) provides the same functions with the
// species, reactants and stoichiometry as constants; both read the rate
// constants from the kernel parameters. Z: the model has order-0 reactions.
template <bool Z>
struct RtModel {
    static constexpr bool kGlobalTrial = false;  // trial counts in shared memory
    static constexpr bool kExpLeave = false;     // the EULER leave law (species scale in shared memory)
    __device__ static int S(const ModelDev &m) { return m.S; }
    __device__ static int R(const ModelDev &m) { return m.R; }
    __device__ static uint32_t diffusive(const ModelDev &m) { return m.diffusive; }
    __device__ static uint32_t need(const RxnTab &tb, int r) { return tb.need[r]; }
    template <int BLOCK>
    __device__ static void build(const ModelDev &m, RxnTab &tb) {
        build_rxn_tab<BLOCK>(m, tb);
    }
    __device__ static float prop(const RxnTab &tb, const ModelDev &, int r, const int32_t *cnt, float inv_nav) {
        return propensity(tb.p[r], cnt, inv_nav, Z);
    }
    // f(species, delta) for each species reaction r changes, in species order
    template <class F>
    __device__ static void for_changes(const RxnTab &tb, int r, F f) {
        const uint4 c = tb.chg[r];
        const int n = tb.nchg[r];
        for (int q = 0; q < n; ++q) {
            const uint32_t sw = q < 4 ? c.x : c.y, dw = q < 4 ? c.z : c.w;
            f((int)((sw >> (8 * (q & 3))) & 0xFFu), (int)(int8_t)((dw >> (8 * (q & 3))) & 0xFFu));
        }
    }
};

// Running sums of the propensities in reaction order, psum[r] = a_0 + ... + a_r
// (inactive reactions contribute 0); returns a_0 + ... + a_{R-1}.
template <class P, int RM>
__device__ __forceinline__ float propensity_sums(const RxnTab &tb, const ModelDev &m, const int32_t *cnt,
                                                 float inv_nav, uint32_t active, float *psum) {
    float a0 = 0.0f;
#pragma unroll
    for (int r = 0; r < RM; ++r) {
        if (r < P::R(m)) {
            const float ar = ((active >> r) & 1u) ? P::prop(tb, m, r, cnt, inv_nav) : 0.0f;
            a0 = __fadd_rn(a0, ar);
            psum[r] = a0;
        }
    }
    return a0;
}

// The last reaction with a positive propensity (the pick when u2 a0 reaches
// every running sum), or -1.
template <class P, int RM>
__device__ __noinline__ int last_positive(const RxnTab &tb, const ModelDev &m, const int32_t *cnt, float inv_nav,
                                          uint32_t active) {
    int last = -1;
#pragma unroll
    for (int r = 0; r < RM; ++r)
        if (r < P::R(m) && ((active >> r) & 1u) && P::prop(tb, m, r, cnt, inv_nav) > 0.0f) last = r;
    return last;
}

// The reaction an event fires: the first r whose running sum exceeds
// target = u2 a0 (running sums only grow, so that is the number of sums
// <= target); if none does, the last reaction with a positive propensity.
template <class P, int RM>
__device__ __forceinline__ int pick_reaction(const RxnTab &tb, const ModelDev &m, const float *psum, float target,
                                             const int32_t *cnt, float inv_nav, uint32_t active) {
    int n = 0;
#pragma unroll
    for (int r = 0; r < RM; ++r)
        if (r < P::R(m)) n += psum[r] <= target ? 1 : 0;
    return n < P::R(m) ? n : last_positive<P, RM>(tb, m, cnt, inv_nav, active);
}

// Stochastic rounding of a mean occupancy: floor(nbar) + [u < nbar - floor(nbar)]
// with u = (w + 1/2) 2^-32. Both the floor and the comparison are exact real
// operations on the double nbar >= 0, evaluated here on its bit pattern with
// integer arithmetic (value = mant 2^-sh): the same result as the double
// operations, without using the FP64 pipe.
__device__ __forceinline__ long long round_trials(double nbar, uint32_t w) {
    const uint64_t bits = (uint64_t)__double_as_longlong(nbar);
    const int e = (int)((bits >> 52) & 0x7ffu);
    if (e == 0 || (bits >> 63)) return 0;  // zero (or negative, not reached): no trials
    const uint64_t mant = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    const int sh = 1075 - e;  // fraction bits of mant
    if (sh <= 0) return (long long)(mant << min(-sh, 10));  // integral (counts are < 2^31)
    long long fl;
    uint64_t f;
    if (sh >= 64) {
        fl = 0;
        f = mant;
    } else {
        fl = (long long)(mant >> sh);
        f = mant & ((1ull << sh) - 1);
    }
    // u < f 2^-sh  <=>  (2w + 1) 2^sh < f 2^33; beyond sh = 90 the fraction is < 2^-38 < u
    if (sh > 90) return fl;
    const unsigned __int128 lhs = (unsigned __int128)(2ull * w + 1ull) << sh;
    const unsigned __int128 rhs = (unsigned __int128)f << 33;
    return fl + (lhs < rhs ? 1 : 0);
}

// Reaction SSA operator for one tet over tau_k (Algorithm 1, reaction part):
// Gillespie's direct method with float propensities and double time, and
// the time-weighted occupancy of every species a fired reaction changes.
// Counts live in shared memory (cnt[s * BLOCK]). The caller has already
// fired the tet's first event (reaction pick0 at time dt0, counts updated);
// this continues from event 1. On return `touched` has a bit for every
// species a fired reaction changed, with its occupancy integral up to its
// last change in O[s] and the time of that change in tS[s]. Returns error
// bits.
template <int BLOCK, int RM, class P>
__device__ uint32_t ssa_tet(const RxnTab &tb, const ModelDev &m, const StepArgs &a, int32_t *cnt, uint32_t tet,
                            uint32_t c0, uint32_t c3, float inv_nav, uint32_t active, int pick0, float dt0, double *O,
                            double *tS, uint32_t &touched) {
    uint32_t bad = 0;
    touched = 0;
    double dt_acc = (double)dt0;  // 0 + (double)dt0: exact
    // occupancy after the first event: O_S = n_before * dt0 (0 + n (dt - 0), both steps exact)
    P::for_changes(tb, pick0, [&](int s, int d) {
        O[s] = __dmul_rn((double)(cnt[s * BLOCK] - d), dt_acc);
        tS[s] = dt_acc;
        touched |= 1u << s;
    });
    uint32_t j = 1;
    for (;;) {
        // keep the reaction table out of registers across iterations
        asm volatile("" ::: "memory");
        // the attempt's two uniforms do not depend on the state: start them first
        const uint4 w = philox4x32_10(a.key0, a.key1, c0, tet, j, (kPurposeReac << 28) | c3);
        const float neg_log_u1 = -steps_logf(unit24f(w.x));
        const float u2 = unit24f(w.y);
        float psum[RM];
        const float a0 = propensity_sums<P, RM>(tb, m, cnt, inv_nav, active, psum);
        if (!(a0 > 0.0f)) break;
        if (j >= kMaxEventsPerWindow) {  // pathological rates: stop and report, never spin
            bad |= 2u;
            break;
        }
        const float dt = __fdiv_rn(neg_log_u1, a0);
        const double dt_new = __dadd_rn(dt_acc, (double)dt);
        if (dt_new > a.tau_k) break;
        ++j;
        const int pick = pick_reaction<P, RM>(tb, m, psum, __fmul_rn(u2, a0), cnt, inv_nav, active);
        if (pick < 0) break;
        dt_acc = dt_new;
        P::for_changes(tb, pick, [&](int s, int d) {
            const int32_t nn = cnt[s * BLOCK];
            if ((touched >> s) & 1u) {
                O[s] = __dadd_rn(O[s], __dmul_rn((double)nn, __dsub_rn(dt_acc, tS[s])));
            } else {
                O[s] = __dmul_rn((double)nn, dt_acc);  // 0 + n (dt - 0): both steps exact
            }
            tS[s] = dt_acc;
            touched |= 1u << s;
            cnt[s * BLOCK] = nn + d;
        });
    }
    return bad;
}

// Trial count of species s of a tet with end count N (Algorithm 1, diffusion
// operator): N if no reaction changed s (its occupancy is N over the whole
// window) or in END mode; else the mean occupancy
// Nbar = (O_S + N_S (tau - t_S)) / tau, stochastically rounded with word
// s mod 4 of the tet's ROUND block s / 4, clamped to N.
__device__ __forceinline__ int32_t trial_count(const StepArgs &a, int s, int32_t N, bool changed, const double *O,
                                               const double *tS, uint32_t key_tet, uint32_t c0, uint32_t c3,
                                               uint32_t &rblk, uint4 &rb) {
    if (!changed || !a.occ) return N;
    const double occ = __dadd_rn(O[s], __dmul_rn((double)N, __dsub_rn(a.tau_k, tS[s])));
    const double nbar = __dmul_rn(occ, a.inv_tau_k);
    if ((uint32_t)(s >> 2) != rblk) {
        rblk = (uint32_t)(s >> 2);
        rb = philox4x32_10(a.key0, a.key1, c0, key_tet, rblk, (kPurposeRound << 28) | c3);
    }
    const long long mm = round_trials(nbar, word_of(rb, s & 3));
    return mm > N ? N : (int32_t)mm;
}

// The species factor of tet i's thresholds: the window's species scale R_s
// (EULER), or the tet's own leave value L_{s,i} from the EXP table (the
// tet's factor A is then its cumulative face shares).
template <class P>
__device__ __forceinline__ uint32_t species_R(const StepArgs &a, const uint32_t *s_scale, int s, int64_t i) {
    if constexpr (P::kExpLeave) return __ldg(a.leave + (size_t)s * (size_t)a.Tpad + (size_t)i);
    else return s_scale[s];
}

// Leave thresholds of one species: T_f = (A_f R_s) >> 31 (2^31 fixed point).
__device__ __forceinline__ void species_thresholds(const uint4 &A, uint32_t R, uint32_t &T0, uint32_t &T1,
                                                   uint32_t &T2, uint32_t &T3) {
    T0 = (uint32_t)(((uint64_t)A.x * R) >> 31);
    T1 = (uint32_t)(((uint64_t)A.y * R) >> 31);
    T2 = (uint32_t)(((uint64_t)A.z * R) >> 31);
    T3 = (uint32_t)(((uint64_t)A.w * R) >> 31);
}

// One threshold comparison x < T over a group of 32 molecules, one bit plane
// at a time (plane k carries bit 30 - k of every molecule's x, bit j of the
// word for molecule j): where the plane's bit of x differs from T's, the
// comparison is decided (x < T where x has 0 and T has 1); it stays open
// while they agree. und: molecules still open; lt: decided x < T.
__device__ __forceinline__ void plane_compare(uint32_t T, int sh, uint32_t R, uint32_t &und, uint32_t &lt) {
    const uint32_t tb = 0u - ((T >> sh) & 1u);  // all ones where T's bit is 1
    lt |= und & ~R & tb;
    und &= ~(R ^ tb);
}

// Diffusion draws of a species with M >= kBulkMin trial molecules in one tet
// (Algorithm 1, diffusion operator): each trial molecule compares a uniform
// 31-bit x with the cumulative thresholds T_0..T_3 and goes through the
// first face f with x < T_f (stays if x >= T_3), exactly as one word per
// molecule would, but x is assembled from bit planes: groups of 32
// molecules take the words of Philox blocks (window, tet, g << 3 | blk,
// bulk purpose | species << 23 | window high bits), plane k = word k of the
// group. Planes are drawn only until every comparison of the group is
// decided (a comparison still open after all 31 planes has x = T: not less).
// The movers go to the neighbours' entries of nxt, one atomic add per face;
// returns how many left.
__device__ __forceinline__ int32_t bulk_species(const StepArgs &a, int32_t *nxt, int s, int32_t M, const uint4 A,
                                             uint32_t Rs, const int4 nb, uint32_t key_tet, uint32_t c0, uint32_t c3) {
    uint32_t T0, T1, T2, T3;
    species_thresholds(A, Rs, T0, T1, T2, T3);
    const uint32_t c3b = (kPurposeBulk << 28) | ((uint32_t)s << 23) | (c3 & 0x007FFFFFu);
    int32_t n0 = 0, n1 = 0, n2 = 0, n3 = 0;
    for (uint32_t g = 0; 32u * g < (uint32_t)M; ++g) {
        const uint32_t m = min(32u, (uint32_t)M - 32u * g);
        const uint32_t valid = m == 32u ? 0xFFFFFFFFu : (1u << m) - 1u;
        // T_f = 2^31: every x < T_f; T_f = 0: none
        uint32_t l0 = T0 >= 0x80000000u ? valid : 0u, u0 = (T0 >= 0x80000000u || T0 == 0u) ? 0u : valid;
        uint32_t l1 = T1 >= 0x80000000u ? valid : 0u, u1 = (T1 >= 0x80000000u || T1 == 0u) ? 0u : valid;
        uint32_t l2 = T2 >= 0x80000000u ? valid : 0u, u2 = (T2 >= 0x80000000u || T2 == 0u) ? 0u : valid;
        uint32_t l3 = T3 >= 0x80000000u ? valid : 0u, u3 = (T3 >= 0x80000000u || T3 == 0u) ? 0u : valid;
        for (uint32_t blk = 0; blk < 8u && (u0 | u1 | u2 | u3); ++blk) {
            const uint4 r = philox4x32_10(a.key0, a.key1, c0, key_tet, (g << 3) | blk, c3b);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = 4 * (int)blk + q;
                if (k <= 30) {
                    const uint32_t R = word_of(r, (uint32_t)q);
                    const int sh = 30 - k;
                    plane_compare(T0, sh, R, u0, l0);
                    plane_compare(T1, sh, R, u1, l1);
                    plane_compare(T2, sh, R, u2, l2);
                    plane_compare(T3, sh, R, u3, l3);
                }
            }
        }
        // cumulative thresholds: l0 within l1 within l2 within l3
        n0 += __popc(l0);
        n1 += __popc(l1 & ~l0);
        n2 += __popc(l2 & ~l1);
        n3 += __popc(l3 & ~l2);
    }
    int32_t *row = nxt + (size_t)s * (size_t)a.Tpad;
    if (n0) atomicAdd(row + nb.x, n0);
    if (n1) atomicAdd(row + nb.y, n1);
    if (n2) atomicAdd(row + nb.z, n2);
    if (n3) atomicAdd(row + nb.w, n3);
    return n0 + n1 + n2 + n3;
}

// Per-warp work state of the diffusion operator. The warp's chunk holds up
// to 32 tets; their trial molecules form one stream per tet (species in
// order), cut into Philox blocks of 4 words. Block b of the chunk belongs to
// lane `owner` with first[lane] <= b < first[lane + 1]; the map caches the
// owner, the species of the block's first word and the tet's trial
// molecules before that species for the first kMapCap blocks (a program may
// set a smaller map to fit more resident blocks; blocks past it are found by
// search).
#ifndef STEPS_MAP_CAP
#define STEPS_MAP_CAP 160
#endif
constexpr int kMapCap = STEPS_MAP_CAP;

struct WarpWork {
    int16_t tet[32];          // tile index of each lane's tet (-1: none)
    uint32_t hm[32];          // species with trial molecules
    uint32_t W[32];           // trial molecules (words) of the tet
    uint32_t touched[32];     // species its reactions changed
    uint32_t first[33];       // exclusive prefix of the lanes' block counts
    uint32_t map[kMapCap];    // lane | species << 5 | block-in-tet << 10 | words before the species << 17
};
// A tet's word stream holds fewer than kBulkMin trial molecules of each
// species, so a block index fits the map's 7 bits and a word offset its 15.
static_assert((kBulkMin - 1) * kMaxSpecies <= 4 * 128, "block-in-tet field of the map");

// One Philox block (4 words) of a tet's diffusion stream: word w decides
// trial molecule w (species in order): face f when T_{f-1} <= x < T_f with
// x = w >> 1 and cumulative thresholds T, stay when x >= T_3. A mover is
// added to the neighbour's entry of nxt and removed from the tet's count.
template <int BLOCK, class P>
__device__ __forceinline__ void diffuse_block(const StepArgs &a, int32_t *nxt, const WarpWork &ww, uint32_t item,
                                              const int32_t *trial_all, size_t tstride, int32_t *cnt_all,
                                              const uint4 *s_thr,
                                              const int4 *s_nbr, const uint32_t *s_tet, const uint32_t *s_scale,
                                              uint32_t c0, uint32_t c3, int64_t i0) {
    int lane, s;
    uint32_t k, before;
    if (item < (uint32_t)kMapCap) {
        const uint32_t o = ww.map[item];
        lane = (int)(o & 31u);
        s = (int)((o >> 5) & 31u);
        k = (o >> 10) & 127u;
        before = o >> 17;
    } else {
        // the owner: last lane with first[lane] <= item; the species: walk the tet's
        // species until the block's first word
        int lo = 0, hi = 31;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (ww.first[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        lane = lo;
        k = item - ww.first[lane];
        const int t = ww.tet[lane];
        uint32_t hm = ww.hm[lane];
        s = __ffs(hm) - 1;
        before = 0;
        uint32_t end = (uint32_t)trial_all[s * tstride + t];
        while (4u * k >= end) {
            hm &= hm - 1;
            s = __ffs(hm) - 1;
            before = end;
            end += (uint32_t)trial_all[s * tstride + t];
        }
    }
    const int t = ww.tet[lane];
    const uint32_t Wt = ww.W[lane];
    uint32_t hm = ww.hm[lane] & ~((2u << s) - 1u);  // species after s
    uint32_t end = before + (uint32_t)trial_all[s * tstride + t];
    const uint4 A = s_thr[t];
    const int4 nb = s_nbr[t];
    const size_t Tpad = (size_t)a.Tpad;
    const uint4 rw = philox4x32_10(a.key0, a.key1, c0, s_tet[t], k, (kPurposeDiff << 28) | c3);
    uint32_t T0, T1, T2, T3;
    species_thresholds(A, species_R<P>(a, s_scale, s, i0 + t), T0, T1, T2, T3);
    uint32_t w = 4u * k;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (w < Wt) {
            if (w >= end) {  // next species with trial molecules
                s = __ffs(hm) - 1;
                hm &= hm - 1;
                end += (uint32_t)trial_all[s * tstride + t];
                species_thresholds(A, species_R<P>(a, s_scale, s, i0 + t), T0, T1, T2, T3);
            }
            const uint32_t x = word_of(rw, q) >> 1;
            if (x < T3) {
                const int nbr = x < T0 ? nb.x : x < T1 ? nb.y : x < T2 ? nb.z : nb.w;
                atomicAdd(nxt + s * Tpad + nbr, 1);
                atomicSub(&cnt_all[s * BLOCK + t], 1);
            }
            ++w;
        }
    }
}

// What stays in tet t after diffusion is added to its own entry of nxt. Every
// entry of nxt is zero when the window starts (the previous window zeroed the
// non-zero entries of this buffer as it read them; set-up zeroes it once), so
// only non-zero counts are written: an immobile species by this tet alone, a
// mobile one by an atomic add beside the movers from the neighbours. `may`
// holds the species that can be non-zero (non-zero at the start or changed by
// a reaction).
template <int BLOCK, class P>
__device__ __forceinline__ void apply_remaining(const ModelDev &m, const StepArgs &a, int32_t *nxt,
                                                const int32_t *cnt_all, int t, uint32_t may, int64_t i0) {
    int32_t *out = nxt + i0 + t;
    const size_t Tpad = (size_t)a.Tpad;
    while (may) {
        const int s = __ffs(may) - 1;
        may &= may - 1;
        const int32_t N = cnt_all[s * BLOCK + t];
        if (N) {
            if ((P::diffusive(m) >> s) & 1u) atomicAdd(out + s * Tpad, N);
            else out[s * Tpad] = N;
        }
    }
}


__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Called by one whole warp: waits until every neighbour tile of tile t has
// published tile_done >= need (acquire loads, one neighbour per lane), for at
// most `limit` cycles (by default 2^31, about a second; false on timeout). A
// finished tile is published by its thread 0 with a release store after the
// block's barrier; lane 0 then orders the tile's bulk copies (async proxy)
// after these loads.
__device__ __forceinline__ bool flow_deps_wait(const FlowArgs &f, uint32_t t, uint32_t need,
                                               long long limit = 2ll << 30) {
    const int lane = threadIdx.x & 31;
    const int b0 = f.tnb_off[t], b1 = f.tnb_off[t + 1];
    const long long t0 = clock64();
    bool ok = true;
    for (int base = b0; base < b1 && ok; base += 32) {
        const int j = base + lane;
        const uint32_t *p = j < b1 ? f.tile_done + f.tnb[j] : nullptr;
        for (;;) {
            const bool done = !p || (int32_t)(ld_acquire_gpu(p) - need) >= 0;
            if (__all_sync(0xFFFFFFFFu, done)) break;
            if (__any_sync(0xFFFFFFFFu, clock64() - t0 > limit)) {
                ok = false;
                break;
            }
            __nanosleep(64);
        }
    }
    __syncwarp();
    if (lane == 0) asm volatile("fence.proxy.async.global;" ::: "memory");
    return ok;
}

// One diffusion window for BLOCK consecutive tets (device order).
//  load   counts and tables into shared memory by bulk copies; each thread
//         notes its tet's non-zero species and zeroes their entries in `cur`
//         (which receives the window after next)
//  A      each thread: its tet's propensities (reactions no tet of the warp
//         can fire are skipped warp-wide: their propensity is 0) and first
//         waiting time, in float; (double)dt > tau_k is tested as
//         dt > tau_dn, tau_dn the largest float <= tau_k (the same decision);
//         a tet whose first event falls inside the window fires it here and
//         is listed as reacting, the others holding molecules as calm
//  chunks each warp takes chunks of 32 listed tets (reacting tets first):
//         the reacting tets' SSA from their second event on; trial counts;
//         the chunk's Philox blocks of trial words (each word moves or keeps
//         one trial molecule; movers are added to the neighbour's entry of
//         `nxt` at once), spread over the warp's lanes for calm chunks and
//         over the whole block, after a barrier, for chunks with reacting
//         tets; then each tet's remaining counts are added to its own entry
//         of `nxt`. Z: the model has order-0 reactions.
// FLOW (a launch of several windows): 1, the block takes its item (window
// q, tile) from f's counter (flow_tiles); 2, the caller took it and passes q
// and the tile's index among f's tiles, dep (batch_flow_tile). Tile `tile`
// of window a.window + q then waits for the tiles listed for dep and
// publishes dep when done. Returns false when the tile's copies or the tiles
// it depends on did not arrive within the wait limits.
template <int BLOCK, int RM, class P, int FLOW = 0>
__device__ __forceinline__ bool step_tile(const ModelDev &m, const StepArgs &a, int64_t tile,
                                          const FlowArgs *f = nullptr, uint32_t q = 0, uint32_t dep = 0) {
    extern __shared__ __align__(16) int32_t smem[];  // cnt [S + 1][BLOCK], trial [S][BLOCK]
    __shared__ __align__(16) uint4 s_thr[BLOCK];
    __shared__ __align__(16) int4 s_nbr[BLOCK];
    __shared__ __align__(16) uint32_t s_tet[BLOCK];
    __shared__ __align__(16) float s_inv_nav[BLOCK];
    __shared__ __align__(16) uint32_t s_mask[BLOCK];
    __shared__ uint32_t s_nz[BLOCK];      // species with a non-zero count at window start
    __shared__ int16_t list[BLOCK];       // reacting tets from the front, calm tets from the back
    __shared__ float q_dt[BLOCK];         // time of a reacting tet's first event
    __shared__ int8_t q_pick[BLOCK];      // its reaction
    __shared__ int32_t nreact, ncalm;
    __shared__ uint32_t next_chunk;
    __shared__ WarpWork wwork[BLOCK / 32];
    __shared__ RxnTab tb;
    __shared__ uint32_t s_scale[kMaxSpecies];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_item;

    const int S = P::S(m);
    const int tid = threadIdx.x;
    const int lane = tid & 31;

    // Programmatic dependent launch: the next window's grid may start its
    // blocks as soon as every block of this one has started; they run up to
    // griddepcontrol.wait below (set-up and the copies of the constant tables)
    // while this grid drains. Without such a launch both are no-ops.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    if (tid == 0) {
        nreact = 0;
        ncalm = 0;
        next_chunk = 0;
        mbar_init(&bar, 1);
        if constexpr (FLOW == 1) s_item = atomicAdd(f->fetch, 1u);
    }
    P::template build<BLOCK>(m, tb);
    if (tid < S) s_scale[tid] = a.scale[tid];
    __syncthreads();
    // the window of this tile: q windows after a.window (buffers swapped when q is odd)
    if constexpr (FLOW == 1) {
        const uint32_t item = s_item;
        if (item >= f->nwin * f->ntiles) return true;
        q = item / f->ntiles;
        tile = (int64_t)(item - q * f->ntiles);
        dep = (uint32_t)tile;
    }
    int32_t *const cur = (q & 1u) ? a.nxt : a.cur;
    int32_t *const nxt = (q & 1u) ? a.cur : a.nxt;
    const int64_t i0 = tile * BLOCK;
    const int64_t i = i0 + tid;
    const int nlive = (int)min((int64_t)BLOCK, (int64_t)a.T - i0);
    const bool live = tid < nlive;
    int32_t *cnt_all = smem;                              // rows 0..S-1 counts, row S ones
    // trial counts [S][tstride]: after the count rows in shared memory, or (for
    // models with many species, to leave room for more resident blocks) the
    // tile's columns of a global buffer
    constexpr bool GT = P::kGlobalTrial;
    int32_t *trial_all = GT ? a.trial + i0 : smem + (size_t)(S + 1) * BLOCK;
    const size_t tstride = GT ? (size_t)a.Tpad : (size_t)BLOCK;
    uint32_t c0, c3;  // RNG counter words of the window, set once the previous window is done
    const size_t Tpad = (size_t)a.Tpad;
    uint32_t bad = 0;

    // ---- load: the block's tile of every table, by TMA bulk copies into
    // shared memory (rows padded to 16 bytes; the tables are padded to Tpad)
    if (tid == 0) {
        const uint32_t n4 = ((uint32_t)nlive + 3u) & ~3u;
        const uint32_t bytes = (uint32_t)S * n4 * 4u + 2u * (uint32_t)nlive * 16u + n4 * 4u +
                               (a.orig ? n4 * 4u : 0u) + (a.rmask ? n4 * 4u : 0u);
        mbar_expect_tx(&bar, bytes);
        // the tables no window writes
        bulk_g2s(s_thr, a.thr + i0, (uint32_t)nlive * 16u, &bar);
        bulk_g2s(s_nbr, a.nbr + i0, (uint32_t)nlive * 16u, &bar);
        bulk_g2s(s_inv_nav, a.inv_nav + i0, n4 * 4u, &bar);
        if (a.orig) bulk_g2s(s_tet, a.orig + i0, n4 * 4u, &bar);
        if (a.rmask) bulk_g2s(s_mask, a.rmask + i0, n4 * 4u, &bar);
    }
    if (!a.orig) s_tet[tid] = (uint32_t)i;
    if (!a.rmask) s_mask[tid] = 0xFFFFFFFFu;
    cnt_all[S * BLOCK + tid] = 1;
    // the counts and the window index come from the previous window: wait for
    // it to complete (and its memory to be visible); in a flow launch, for the
    // tiles this one depends on
    bool deps = true;
    if constexpr (FLOW != 0) {
        if (q > 0 && tid < 32) deps = flow_deps_wait(*f, dep, (uint32_t)(a.window + q));
    } else {
        asm volatile("griddepcontrol.wait;" ::: "memory");
    }
    {
        const uint64_t window = a.window + q + (a.window_base ? *a.window_base : 0ull);
        c0 = (uint32_t)window;
        c3 = (uint32_t)(window >> 32) & 0x0FFFFFFFu;
    }
    if (tid == 0) {
        const uint32_t n4 = ((uint32_t)nlive + 3u) & ~3u;
        for (int s = 0; s < S; ++s) bulk_g2s(cnt_all + s * BLOCK, cur + s * Tpad + i0, n4 * 4u, &bar);
        // the tile `prefetch` tiles ahead, processed about half a resident
        // wave later, into L2. The last wave's blocks take the next window's first
        // tiles, from the buffer that window reads (lines that this window's
        // atomics still change are only brought into L2, where they land).
        int64_t p0 = i0 + (int64_t)a.prefetch * BLOCK;
        const int32_t *pc = cur;
        if (p0 >= a.T) {
            p0 -= ((int64_t)a.T + BLOCK - 1) / BLOCK * BLOCK;
            pc = nxt;
        }
        if (a.prefetch > 0 && p0 >= 0 && p0 < a.T) {
            const uint32_t pl = (uint32_t)min((int64_t)BLOCK, (int64_t)a.T - p0);
            const uint32_t p4 = (pl + 3u) & ~3u;
            for (int s = 0; s < S; ++s) bulk_prefetch_l2(pc + s * Tpad + p0, p4 * 4u);
            bulk_prefetch_l2(a.thr + p0, pl * 16u);
            bulk_prefetch_l2(a.nbr + p0, pl * 16u);
            bulk_prefetch_l2(a.inv_nav + p0, p4 * 4u);
            if (a.orig) bulk_prefetch_l2(a.orig + p0, p4 * 4u);
            if (a.rmask) bulk_prefetch_l2(a.rmask + p0, p4 * 4u);
        }
    }
    // one thread waits for the copies (bounded) while the others sleep at the
    // barrier; then every thread observes the completed phase itself
    bool arrived = true;
    if (tid == 0) arrived = mbar_wait_bounded(&bar, 0);
    if (__syncthreads_or(!arrived || !deps)) {
        // the copies did not land in time (or the tiles this one depends on did
        // not finish): report, let the copies finish (bounded), skip the window
        if (tid == 0) {
            atomicOr(a.err, (arrived ? 0u : 4u) | (deps ? 0u : 8u));
            if (!arrived) mbar_wait_bounded(&bar, 0);
        }
        __syncthreads();
        return false;
    }
    mbar_try_wait(&bar, 0);  // completed: returns at once
    // `cur` receives the window after next: zero its non-zero entries (an
    // immobile entry is overwritten by that window anyway)
    uint32_t nz = 0;
    if (live) {
        int32_t vmin = 0;
        int32_t *row = cur + i;
#pragma unroll 4
        for (int s = 0; s < S; ++s) {
            const int32_t v = cnt_all[s * BLOCK + tid];
            vmin = min(vmin, v);
            if (v != 0) {
                nz |= 1u << s;
                *row = 0;
            }
            row += Tpad;
        }
        bad |= vmin < 0 ? 1u : 0u;
    }
    s_nz[tid] = nz;

    // ---- A: the tet's first reaction event, if it falls inside the window
    bool reacting = false;
    if (P::R(m) > 0) {
        const float inv_nav = s_inv_nav[tid];
        const uint32_t active = live ? s_mask[tid] : 0u;
        int32_t *cnt = cnt_all + tid;
        float psum[RM];
        float a0 = 0.0f;
        // a_r = 0 (exactly: a product with a zero count) unless every reactant
        // is present; reactions no tet of the warp can fire are skipped
        // lane r decides whether reaction r can fire in any tet of the warp
        const uint32_t wnz = __reduce_or_sync(0xFFFFFFFFu, nz);
        const uint32_t wact = __reduce_or_sync(0xFFFFFFFFu, active);
        const uint32_t need_l = lane < P::R(m) ? P::need(tb, lane) : 0u;
        const uint32_t possible =
            __ballot_sync(0xFFFFFFFFu, lane < P::R(m) && ((wact >> lane) & 1u) && (wnz & need_l) == need_l);
        if (possible) {
#pragma unroll
            for (int r = 0; r < RM; ++r) {
                if (r < P::R(m)) {
                    float ar = 0.0f;
                    if ((possible >> r) & 1u)
                        ar = ((active >> r) & 1u) ? P::prop(tb, m, r, cnt, inv_nav) : 0.0f;
                    a0 = __fadd_rn(a0, ar);
                    psum[r] = a0;
                }
            }
        }
        if (live && a0 > 0.0f) {
            const uint4 w = philox4x32_10(a.key0, a.key1, c0, s_tet[tid], 0u, (kPurposeReac << 28) | c3);
            const float dt = __fdiv_rn(-steps_logf(unit24f(w.x)), a0);
            // 0 + (double)dt is exact, and (double)dt > tau_k <=> dt > tau_dn
            if (!(dt > a.tau_dn)) {
                const int pick = pick_reaction<P, RM>(tb, m, psum, __fmul_rn(unit24f(w.y), a0), cnt, inv_nav,
                                                      active);
                if (pick >= 0) {
                    P::for_changes(tb, pick, [&](int s, int d) { cnt[s * BLOCK] += d; });
                    q_pick[tid] = (int8_t)pick;
                    q_dt[tid] = dt;
                    reacting = true;
                }
            }
        }
    }
    {
        // warp-aggregated list appends: one atomic per warp and list
        // a calm tet with no molecules has nothing to do this window
        const uint32_t rmask = __ballot_sync(0xFFFFFFFFu, live && reacting);
        const uint32_t cmask = __ballot_sync(0xFFFFFFFFu, live && !reacting && nz != 0u);
        int rbase = 0, cbase = 0;
        if (lane == 0) {
            if (rmask) rbase = atomicAdd(&nreact, __popc(rmask));
            if (cmask) cbase = atomicAdd(&ncalm, __popc(cmask));
        }
        rbase = __shfl_sync(0xFFFFFFFFu, rbase, 0);
        cbase = __shfl_sync(0xFFFFFFFFu, cbase, 0);
        const uint32_t below = (1u << lane) - 1u;
        if ((rmask >> lane) & 1u) list[rbase + __popc(rmask & below)] = (int16_t)tid;
        else if ((cmask >> lane) & 1u) list[BLOCK - 1 - (cbase + __popc(cmask & below))] = (int16_t)tid;
    }
    __syncthreads();

    // ---- phase 1: chunks of 32 listed tets (reacting tets first, then calm
    // ones), one warp each. The reacting chunks run their SSA and trial counts
    // and leave their diffusion to phase 2; calm chunks finish here.
    const int nr = nreact, nc = ncalm;
    const int nchunks = (nr + nc + 31) >> 5;
    const int rchunks = (nr + 31) >> 5;
    for (;;) {
        uint32_t ch = 0;
        if (lane == 0) ch = atomicAdd(&next_chunk, 1u);
        ch = __shfl_sync(0xFFFFFFFFu, ch, 0);
        if (ch >= (uint32_t)nchunks) break;
        WarpWork &ww = wwork[ch];
        const int j = (int)ch * 32 + lane;  // position in [reacting..., calm...]
        const bool valid = j < nr + nc;
        const bool reacts = j < nr;
        const int t = !valid ? -1 : reacts ? list[j] : list[BLOCK - 1 - (j - nr)];

        // the reacting tets' SSA from their second event on
        uint32_t touched = 0;
        double O[kMaxSpecies], tS[kMaxSpecies];
        if (reacts)
            bad |= ssa_tet<BLOCK, RM, P>(tb, m, a, cnt_all + t, s_tet[t], c0, c3, s_inv_nav[t], s_mask[t],
                                         q_pick[t], q_dt[t], O, tS, touched);

        // trial counts: species that may hold molecules (non-zero at the start, or
        // changed by a reaction), diffusive, with a non-zero leave threshold.
        // Species with kBulkMin or more trial molecules draw by bit planes here
        // (their movers leave at once); the others join the tet's word stream.
        uint32_t W = 0, hm = 0, bm = 0;
        if (valid) {
            uint32_t walk = (s_nz[t] | touched) & P::diffusive(m);
            const uint32_t Aw = s_thr[t].w;
            // one loop for lanes with and without occupancy rounding (a reacting
            // chunk holds both); without it the trial count is the count
            const bool plain = !touched || !a.occ;
            uint32_t rblk = 0xFFFFFFFFu;
            uint4 rb = make_uint4(0, 0, 0, 0);
            while (walk) {
                const int s = __ffs(walk) - 1;
                walk &= walk - 1;
                if ((uint32_t)(((uint64_t)Aw * species_R<P>(a, s_scale, s, i0 + t)) >> 31) == 0u)
                    continue;  // draws nothing
                const int32_t N = cnt_all[s * BLOCK + t];
                const int32_t M = plain ? N
                                        : trial_count(a, s, N, (touched >> s) & 1u, O, tS, s_tet[t], c0, c3, rblk, rb);
                if (M > 0) {
                    trial_all[s * tstride + t] = M;
                    if (M >= kBulkMin) {
                        bm |= 1u << s;
                    } else {
                        hm |= 1u << s;
                        W += (uint32_t)M;
                    }
                }
            }
        }
        // species with many trial molecules: bit-plane draws by the lane that
        // owns the tet, movers sent now (they are rare unless counts are high,
        // and then every lane has some). The warp walks the union of its lanes'
        // bulk species in species order, so that the lanes drawing for one
        // species (similar counts, the same thresholds' scale) run together.
        uint32_t bw = __reduce_or_sync(0xFFFFFFFFu, bm);
        while (bw) {
            const int s = __ffs(bw) - 1;
            bw &= bw - 1;
            if ((bm >> s) & 1u)
                cnt_all[s * BLOCK + t] -= bulk_species(a, nxt, s, trial_all[s * tstride + t], s_thr[t],
                                                       species_R<P>(a, s_scale, s, i0 + t), s_nbr[t], s_tet[t], c0, c3);
        }
        // the chunk's Philox blocks: exclusive prefix of the lanes' block counts
        const uint32_t nb = (W + 3u) >> 2;
        uint32_t x = nb;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
            if (lane >= d) x += y;
        }
        const uint32_t first = x - nb;
        const uint32_t total = __shfl_sync(0xFFFFFFFFu, x, 31);
        ww.tet[lane] = (int16_t)t;
        ww.hm[lane] = hm;
        ww.W[lane] = W;
        ww.touched[lane] = touched;
        ww.first[lane] = first;
        if (lane == 31) ww.first[32] = total;
        if (nb > 0 && first < (uint32_t)kMapCap) {
            int s = __ffs(hm) - 1;
            uint32_t h = hm & (hm - 1), before = 0, end = (uint32_t)trial_all[s * tstride + t];
            for (uint32_t k = 0; k < nb && first + k < (uint32_t)kMapCap; ++k) {
                while (4u * k >= end) {
                    s = __ffs(h) - 1;
                    h &= h - 1;
                    before = end;
                    end += (uint32_t)trial_all[s * tstride + t];
                }
                ww.map[first + k] = (uint32_t)lane | ((uint32_t)s << 5) | (k << 10) | (before << 17);
            }
        }
        __syncwarp();
        if (ch < (uint32_t)rchunks) continue;  // diffusion in phase 2
        for (uint32_t item = lane; item < total; item += 32)
            diffuse_block<BLOCK, P>(a, nxt, ww, item, trial_all, tstride, cnt_all, s_thr, s_nbr, s_tet, s_scale, c0, c3, i0);
        __syncwarp();
        if (valid) apply_remaining<BLOCK, P>(m, a, nxt, cnt_all, t, s_nz[t] | touched, i0);
        __syncwarp();
    }

    // ---- phase 2: the reacting chunks' Philox blocks, spread over the block;
    // phase 3: their tets' remaining counts
    if (rchunks > 0) {
        __syncthreads();
        for (int c = 0; c < rchunks; ++c) {
            const WarpWork &ww = wwork[c];
            const uint32_t total = ww.first[32];
            for (uint32_t item = tid; item < total; item += BLOCK)
                diffuse_block<BLOCK, P>(a, nxt, ww, item, trial_all, tstride, cnt_all, s_thr, s_nbr, s_tet, s_scale, c0, c3, i0);
        }
        __syncthreads();
        for (int c = tid >> 5; c < rchunks; c += BLOCK / 32) {
            const int t = wwork[c].tet[lane];
            if (t >= 0) apply_remaining<BLOCK, P>(m, a, nxt, cnt_all, t, s_nz[t] | wwork[c].touched[lane], i0);
        }
    }
    if (bad) atomicOr(a.err, bad);
    if constexpr (FLOW != 0) {
        // publish: every thread's writes of this tile come before the release
        __syncthreads();
        if (tid == 0) st_release_gpu(f->tile_done + dep, (uint32_t)(a.window + q + 1));
    }
    return true;
}

// Full windows of one simulation in one launch of nwin x ntiles blocks. Each
// block takes the next item (window q, tile t), q-major, from a counter. The
// item (q, t) with q > 0 waits until every tile that shares a face with t,
// and t itself, has finished window q - 1: the counts t reads are then
// complete (every atomic that adds into them has landed), and the entries of
// the buffer t adds into have been read and zeroed by their own tiles. Those
// are all the dependencies of a window's tile (Algorithm 1: a tet's new
// counts come from itself and its face neighbours only), so a window's first
// tiles start while the previous window's last tiles still run, with no
// grid-wide boundary between windows. An item waits only on items taken
// before it, which running blocks hold, so the items complete whatever the
// number of resident blocks.
template <int BLOCK, int RM, class P>
__device__ __forceinline__ void flow_tiles(const ModelDev &m, const StepArgs &a, const FlowArgs &f) {
    step_tile<BLOCK, RM, P, 1>(m, a, 0, &f);
}

// One block of a batched launch: the member named by work[blockIdx.x] copies
// its model and window arguments from the device table into shared memory
// (cur/nxt by the member's buffer parity) and runs the tile body. A member
// whose windows are done returns at once (block-uniform).
template <int BLOCK, int RM, class P>
__device__ __forceinline__ void batch_tile(const BlockWork *__restrict__ work, const RepEntry *__restrict__ reps,
                                           int32_t prefetch) {
    __shared__ __align__(16) ModelDev t_model;
    __shared__ __align__(16) StepArgs t_args;
    __shared__ int32_t t_tile;
    const BlockWork bw = work[blockIdx.x];
    const RepEntry *e = reps + bw.rep;
    if (e->args.window >= e->window_end) return;
    static_assert(sizeof(ModelDev) % 4 == 0 && sizeof(StepArgs) % 4 == 0, "word copy");
    const uint32_t *src_m = reinterpret_cast<const uint32_t *>(&e->model);
    uint32_t *dst_m = reinterpret_cast<uint32_t *>(&t_model);
    for (int k = threadIdx.x; k < (int)(sizeof(ModelDev) / 4); k += BLOCK) dst_m[k] = src_m[k];
    const uint32_t *src_a = reinterpret_cast<const uint32_t *>(&e->args);
    uint32_t *dst_a = reinterpret_cast<uint32_t *>(&t_args);
    for (int k = threadIdx.x; k < (int)(sizeof(StepArgs) / 4); k += BLOCK) dst_a[k] = src_a[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        t_args.cur = e->cnt[e->parity];
        t_args.nxt = e->cnt[e->parity ^ 1u];
        t_args.prefetch = prefetch;  // tiles ahead within the member
        t_tile = bw.tile;
    }
    __syncthreads();
    step_tile<BLOCK, RM, P>(t_model, t_args, (int64_t)t_tile);
}

// Full windows of a group of batch members in one launch (the batched form of
// flow_tiles). The group's tiles are work[work0 .. work0 + f.ntiles), member
// by member; item (q, i) is tile work0 + i of window q of its member (its own
// window index and buffers). A member whose windows end earlier skips its
// later items; nothing depends on them (the dependencies stay within a
// member). f's tile lists and words are indexed by work entry.
template <int BLOCK, int RM, class P>
__device__ __forceinline__ void batch_flow_tile(const BlockWork *__restrict__ work, const RepEntry *__restrict__ reps,
                                                const FlowArgs &f, uint32_t work0, int32_t prefetch) {
    __shared__ __align__(16) ModelDev t_model;
    __shared__ __align__(16) StepArgs t_args;
    __shared__ uint32_t s_q, s_dep;
    __shared__ int32_t s_rep, s_tile;
    if (threadIdx.x == 0) {
        const uint32_t item = atomicAdd(f.fetch, 1u);
        s_rep = -1;
        if (item < f.nwin * f.ntiles) {
            const uint32_t q = item / f.ntiles, i = item - q * f.ntiles;
            const BlockWork bw = work[work0 + i];
            if (reps[bw.rep].args.window + q < reps[bw.rep].window_end) {
                s_rep = bw.rep;
                s_tile = bw.tile;
                s_q = q;
                s_dep = work0 + i;
            }
        }
    }
    __syncthreads();
    if (s_rep < 0) return;
    const RepEntry *e = reps + s_rep;
    static_assert(sizeof(ModelDev) % 4 == 0 && sizeof(StepArgs) % 4 == 0, "word copy");
    const uint32_t *src_m = reinterpret_cast<const uint32_t *>(&e->model);
    uint32_t *dst_m = reinterpret_cast<uint32_t *>(&t_model);
    for (int k = threadIdx.x; k < (int)(sizeof(ModelDev) / 4); k += BLOCK) dst_m[k] = src_m[k];
    const uint32_t *src_a = reinterpret_cast<const uint32_t *>(&e->args);
    uint32_t *dst_a = reinterpret_cast<uint32_t *>(&t_args);
    for (int k = threadIdx.x; k < (int)(sizeof(StepArgs) / 4); k += BLOCK) dst_a[k] = src_a[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        t_args.cur = e->cnt[e->parity];
        t_args.nxt = e->cnt[e->parity ^ 1u];
        t_args.prefetch = prefetch;  // tiles ahead within the member
    }
    __syncthreads();
    step_tile<BLOCK, RM, P, 2>(t_model, t_args, (int64_t)s_tile, &f, s_q, s_dep);
}

}  // namespace
}  // namespace steps
