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

#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "steps_internal.h"

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

// bytes: multiple of 16; both addresses 16-byte aligned
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase with the given parity to complete, for at most about
// 2^30 clock cycles (~0.5 s); returns false when the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > (1ll << 30)) return false;
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

// Mass-action propensity in float (order 0: k N_A V; 1: k N; 2: k/(N_A V) N_a N_b;
// dimer: k/(N_A V) N (N-1)).
__device__ __forceinline__ float propensity(const ReacDesc &d, const int32_t *cnt, int stride, float inv_nav) {
    switch (d.type) {
    case kOrder0:
        return __fdiv_rn(d.k, inv_nav);
    case kOrder1:
        return __fmul_rn(d.k, __int2float_rn(cnt[d.ra * stride]));
    case kOrder2: {
        const float c = __fmul_rn(d.k, inv_nav);
        return __fmul_rn(__fmul_rn(c, __int2float_rn(cnt[d.ra * stride])), __int2float_rn(cnt[d.rb * stride]));
    }
    default: {
        const float c = __fmul_rn(d.k, inv_nav);
        const int32_t n = cnt[d.ra * stride];
        return __fmul_rn(__fmul_rn(c, __int2float_rn(n)), __int2float_rn(n - 1));
    }
    }
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
// Counts live in shared memory (cnt[s * BLOCK]); on return trial[s * BLOCK]
// holds the integer trial count of every diffusive species the reactions
// changed (mean occupancy, stochastically rounded, clamped to the end count;
// or the end count in END mode). Returns error bits.
template <int BLOCK, int RM>
__device__ uint32_t ssa_tet(const ModelDev &m, const StepArgs &a, int32_t *cnt, int32_t *trial, uint32_t tet,
                            uint32_t c0, uint32_t c3, float inv_nav, uint32_t active) {
    uint32_t touched = 0, bad = 0;
    double O[kMaxSpecies], tS[kMaxSpecies];
    double dt_acc = 0.0;
    uint32_t j = 0;
    for (;;) {
        // keep the model's constants out of registers across iterations (the
        // batched kernel reads them from shared memory)
        asm volatile("" ::: "memory");
        // the attempt's two uniforms do not depend on the state: start them first
        const uint4 w = philox4x32_10(a.key0, a.key1, c0, tet, j, (kPurposeReac << 28) | c3);
        const float neg_log_u1 = -steps_logf(unit24f(w.x));
        const float u2 = unit24f(w.y);
        // propensities; psum[r] = a_0 + ... + a_r summed in reaction order
        float psum[RM];
        uint32_t pos = 0;
        float a0 = 0.0f;
#pragma unroll
        for (int r = 0; r < RM; ++r) {
            if (r < m.R) {
                const float ar = ((active >> r) & 1u) ? propensity(m.reac[r], cnt, BLOCK, inv_nav) : 0.0f;
                a0 = __fadd_rn(a0, ar);
                psum[r] = a0;
                pos |= (ar > 0.0f ? 1u : 0u) << r;
            }
        }
        if (!(a0 > 0.0f)) break;
        if (j >= kMaxEventsPerWindow) {  // pathological rates: stop and report, never spin
            bad |= 2u;
            break;
        }
        const float dt = __fdiv_rn(neg_log_u1, a0);
        double dt_new;
        if (j == 0) {
            // 0 + (double)dt is exact, and (double)dt > tau_k <=> dt > tau_dn
            if (dt > a.tau_dn) break;
            dt_new = (double)dt;
        } else {
            dt_new = __dadd_rn(dt_acc, (double)dt);
            if (dt_new > a.tau_k) break;
        }
        ++j;
        // first reaction whose running sum exceeds u2 a0 (running sums only grow,
        // so the reactions past the target form a suffix); if none, the last
        // reaction with a positive propensity
        const float target = __fmul_rn(u2, a0);
        uint32_t over = 0;
#pragma unroll
        for (int r = 0; r < RM; ++r)
            if (r < m.R) over |= (psum[r] > target ? 1u : 0u) << r;
        const int pick = over ? __ffs(over) - 1 : (pos ? 31 - __clz(pos) : -1);
        if (pick < 0) break;
        dt_acc = dt_new;
        const ReacDesc &d = m.reac[pick];
        for (int q = 0; q < d.nchg; ++q) {
            const int s = d.chg_s[q];
            const int32_t n = cnt[s * BLOCK];
            if ((touched >> s) & 1u) {
                O[s] = __dadd_rn(O[s], __dmul_rn((double)n, __dsub_rn(dt_acc, tS[s])));
            } else {
                O[s] = __dmul_rn((double)n, dt_acc);  // 0 + n (dt - 0): both steps exact
            }
            tS[s] = dt_acc;
            touched |= 1u << s;
            cnt[s * BLOCK] = n + d.chg_d[q];
        }
    }
    // trial counts of the changed diffusive species, one set bit at a time
    uint32_t todo = touched & m.diffusive;
    uint32_t rblk = 0xFFFFFFFFu;
    uint4 rb = make_uint4(0, 0, 0, 0);
    while (todo) {
        const int s = __ffs(todo) - 1;
        todo &= todo - 1;
        const int32_t N = cnt[s * BLOCK];
        int32_t M = N;
        if (a.occ) {
            // Nbar = (O_S + N_S (tau - t_S)) / tau, stochastically rounded, clamped to N_S
            const double occ = __dadd_rn(O[s], __dmul_rn((double)N, __dsub_rn(a.tau_k, tS[s])));
            const double nbar = __dmul_rn(occ, a.inv_tau_k);
            if ((uint32_t)(s >> 2) != rblk) {
                rblk = (uint32_t)(s >> 2);
                rb = philox4x32_10(a.key0, a.key1, c0, tet, rblk, (kPurposeRound << 28) | c3);
            }
            const long long mm = round_trials(nbar, word_of(rb, s & 3));
            M = mm > N ? N : (int32_t)mm;
        }
        trial[s * BLOCK] = M;
    }
    return bad;
}

// Trial words per phase-C work item (two Philox blocks).
constexpr uint32_t kItemWords = 8;

// Block-wide exclusive scan of one value per thread; returns the total.
template <int BLOCK>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *out, uint32_t *warp_tot) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t t = lane < BLOCK / 32 ? warp_tot[lane] : 0u;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, t, d);
            if (lane >= d) t += y;
        }
        if (lane < BLOCK / 32) warp_tot[lane] = t;  // inclusive
    }
    __syncthreads();
    const uint32_t before = wid > 0 ? warp_tot[wid - 1] : 0u;
    out[threadIdx.x] = before + x - v;
    const uint32_t total = warp_tot[BLOCK / 32 - 1];
    return total;
}

// Trial molecules of one tet that draw words: every diffusive species with a
// non-zero leave threshold keeps its trial count, the others get 0 (written
// back to trial[s * stride]). Returns their sum, the tet's word count.
__device__ __forceinline__ uint32_t trial_words(const ModelDev &m, const StepArgs &a, const uint4 A, int32_t *trial,
                                                int stride) {
    uint32_t W = 0;
    for (int s = 0; s < m.S; ++s) {
        int32_t M = 0;
        if ((m.diffusive >> s) & 1u) {
            M = trial[s * stride];
            if ((uint32_t)(((uint64_t)A.w * a.scale[s]) >> 31) == 0u) M = 0;
        }
        trial[s * stride] = M;
        W += (uint32_t)M;
    }
    return W;
}

// Work items per block the item map holds (beyond it, items find their tet
// and species by search).
template <int BLOCK>
struct ItemMap {
    static constexpr uint32_t kCap = 4 * BLOCK;
};

// Fill the item map for this thread's tet t: item blk_start[t] + k covers
// words [k kItemWords, (k+1) kItemWords) of the tet's stream; record the tet,
// the species of the item's first word and the number of the tet's trial
// molecules before that species.
template <int BLOCK>
__device__ __forceinline__ void map_items(int t, uint32_t W, uint32_t first, uint32_t total, const int32_t *trial,
                                          uint32_t *owner, uint32_t *before) {
    if (W == 0 || total > ItemMap<BLOCK>::kCap) return;
    const uint32_t n = (W + kItemWords - 1u) / kItemWords;
    int s = 0;
    uint32_t pre = 0, end = (uint32_t)trial[0];
    for (uint32_t k = 0; k < n; ++k) {
        const uint32_t w = k * kItemWords;
        while (w >= end) {
            pre = end;
            ++s;
            end += (uint32_t)trial[s * BLOCK];
        }
        owner[first + k] = (uint32_t)t | ((uint32_t)s << 9) | (k << 14);
        before[first + k] = pre;
    }
}

// One work item of the diffusion operator: up to kItemWords consecutive words
// of one tet's stream (two Philox blocks), each deciding one trial molecule:
// face f when T_{f-1} <= x < T_f (cumulative thresholds), stay when x >= T_3.
// A mover is added to the neighbour's entry of nxt and removed from this tet's
// shared count.
template <int BLOCK>
__device__ __forceinline__ void diffuse_item(const StepArgs &a, uint32_t item, uint32_t total, int nlive,
                                             const uint32_t *blk_start, const uint32_t *owner,
                                             const uint32_t *before, const uint32_t *words,
                                             const int32_t *trial_all, int32_t *cnt_all, const uint4 *s_thr,
                                             const int4 *s_nbr, const uint32_t *s_tet, uint32_t c0, uint32_t c3) {
    int t, s;
    uint32_t w, end;
    if (total <= ItemMap<BLOCK>::kCap) {
        const uint32_t o = owner[item];
        t = (int)(o & 0x1FFu);
        s = (int)((o >> 9) & 0x1Fu);
        w = (o >> 14) * kItemWords;
        end = before[item] + (uint32_t)trial_all[s * BLOCK + t];
    } else {
        // the tet owning this item: last t with blk_start[t] <= item
        int lo = 0, hi = nlive - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (blk_start[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        t = lo;
        w = (item - blk_start[t]) * kItemWords;
        s = 0;
        end = (uint32_t)trial_all[t];
        while (w >= end) {
            ++s;
            end += (uint32_t)trial_all[s * BLOCK + t];
        }
    }
    const int32_t *trial = trial_all + t;
    const uint32_t Wt = words[t];
    const uint32_t tet = s_tet[t];
    const uint4 A = s_thr[t];
    const int4 nb = s_nbr[t];
    const size_t Tpad = (size_t)a.Tpad;
    // both Philox blocks of the item as independent chains (the second may go unused)
    const uint4 rw0 = philox4x32_10(a.key0, a.key1, c0, tet, w >> 2, (kPurposeDiff << 28) | c3);
    const uint4 rw1 = philox4x32_10(a.key0, a.key1, c0, tet, (w >> 2) + 1u, (kPurposeDiff << 28) | c3);
    uint64_t R = a.scale[s];
    uint32_t T0 = (uint32_t)(((uint64_t)A.x * R) >> 31), T1 = (uint32_t)(((uint64_t)A.y * R) >> 31);
    uint32_t T2 = (uint32_t)(((uint64_t)A.z * R) >> 31), T3 = (uint32_t)(((uint64_t)A.w * R) >> 31);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (w < Wt) {
            if (w >= end) {  // next species with trial molecules
                do {
                    ++s;
                    end += (uint32_t)trial[s * BLOCK];
                } while (w >= end);
                R = a.scale[s];
                T0 = (uint32_t)(((uint64_t)A.x * R) >> 31);
                T1 = (uint32_t)(((uint64_t)A.y * R) >> 31);
                T2 = (uint32_t)(((uint64_t)A.z * R) >> 31);
                T3 = (uint32_t)(((uint64_t)A.w * R) >> 31);
            }
            const uint32_t x = word_of(k < 4 ? rw0 : rw1, k & 3) >> 1;
            if (x < T3) {
                const int nbr = x < T0 ? nb.x : x < T1 ? nb.y : x < T2 ? nb.z : nb.w;
                atomicAdd(a.nxt + s * Tpad + nbr, 1);
                atomicSub(&cnt_all[s * BLOCK + t], 1);
            }
            ++w;
        }
    }
}

// One diffusion window for BLOCK consecutive tets (device order).
//  load   counts into shared memory; mobile entries of `cur` are zeroed as read
//  A      each thread: its tet's propensities and first waiting time, in float;
//         (double)dt > tau_k is tested as dt > tau_dn, tau_dn the largest float
//         <= tau_k (the same decision); tets with an event are queued
//  B      the queued tets' full SSA and trial counts, one queued tet per thread
//  C      trial words of all the block's tets: Philox blocks of four words are
//         spread evenly over the threads; each word moves or keeps one trial
//         molecule; movers are added to the neighbour in `nxt` at once
//  D      what stays is added to the tet's own entry of `nxt` (coalesced)
template <int BLOCK, int RM>
__device__ __forceinline__ void step_tile(const ModelDev &m, const StepArgs &a, const int64_t tile) {
    extern __shared__ __align__(16) int32_t smem[];  // cnt [S][BLOCK], trial [S][BLOCK]
    __shared__ __align__(16) uint4 s_thr[BLOCK];
    __shared__ __align__(16) int4 s_nbr[BLOCK];
    __shared__ __align__(16) uint32_t s_tet[BLOCK];
    __shared__ __align__(16) float s_inv_nav[BLOCK];
    __shared__ __align__(16) uint32_t s_mask[BLOCK];
    __shared__ int32_t queue[BLOCK];
    __shared__ uint32_t blk_start[BLOCK + 1];
    __shared__ uint32_t words[BLOCK];
    __shared__ uint32_t warp_tot[BLOCK / 32];
    __shared__ int32_t nqueue;
    __shared__ uint8_t reacted[BLOCK];  // 1 = queued for the full SSA
    __shared__ uint32_t next_item;
    __shared__ uint32_t item_owner[ItemMap<BLOCK>::kCap];
    __shared__ uint32_t item_before[ItemMap<BLOCK>::kCap];
    __shared__ __align__(8) uint64_t bar;

    const int S = m.S;
    const int tid = threadIdx.x;
    const int64_t i0 = tile * BLOCK;
    const int64_t i = i0 + tid;
    const int nlive = (int)min((int64_t)BLOCK, (int64_t)a.T - i0);
    const bool live = tid < nlive;
    int32_t *cnt_all = smem;
    int32_t *trial_all = smem + (size_t)S * BLOCK;
    const uint64_t window = a.window + (a.window_base ? *a.window_base : 0ull);
    const uint32_t c0 = (uint32_t)window;
    const uint32_t c3 = (uint32_t)(window >> 32) & 0x0FFFFFFFu;
    const size_t Tpad = (size_t)a.Tpad;
    uint32_t bad = 0;

    // ---- load: the block's tile of every table, by TMA bulk copies into
    // shared memory (rows padded to 16 bytes; the tables are padded to Tpad)
    if (tid == 0) {
        nqueue = 0;
        mbar_init(&bar, 1);
    }
    __syncthreads();
    if (tid == 0) {
        const uint32_t n4 = ((uint32_t)nlive + 3u) & ~3u;
        const uint32_t bytes = (uint32_t)S * n4 * 4u + 2u * (uint32_t)nlive * 16u + n4 * 4u +
                               (a.orig ? n4 * 4u : 0u) + (a.rmask ? n4 * 4u : 0u);
        mbar_expect_tx(&bar, bytes);
        for (int s = 0; s < S; ++s) bulk_g2s(cnt_all + s * BLOCK, a.cur + s * Tpad + i0, n4 * 4u, &bar);
        bulk_g2s(s_thr, a.thr + i0, (uint32_t)nlive * 16u, &bar);
        bulk_g2s(s_nbr, a.nbr + i0, (uint32_t)nlive * 16u, &bar);
        bulk_g2s(s_inv_nav, a.inv_nav + i0, n4 * 4u, &bar);
        if (a.orig) bulk_g2s(s_tet, a.orig + i0, n4 * 4u, &bar);
        if (a.rmask) bulk_g2s(s_mask, a.rmask + i0, n4 * 4u, &bar);
    }
    if (!a.orig) s_tet[tid] = (uint32_t)i;
    if (!a.rmask) s_mask[tid] = 0xFFFFFFFFu;
    reacted[tid] = 0;
    const bool arrived = mbar_wait_bounded(&bar, 0);
    if (__syncthreads_or(!arrived)) {
        // the copies did not land in time: report, let them finish (bounded), skip the window
        if (tid == 0) {
            atomicOr(a.err, 4u);
            mbar_wait_bounded(&bar, 0);
        }
        __syncthreads();
        return;
    }
    if (live) {
        for (int s = 0; s < S; ++s) {
            const int32_t v = cnt_all[s * BLOCK + tid];
            bad |= v < 0 ? 1u : 0u;
            trial_all[s * BLOCK + tid] = v;
            if ((m.diffusive >> s) & 1u) a.cur[s * Tpad + i] = 0;  // receives the window after next
        }
    }
    __syncthreads();

    // ---- A: does the tet's first reaction fall inside the window?
    if (live && m.R > 0) {
        const float inv_nav = s_inv_nav[tid];
        const uint32_t active = s_mask[tid];
        const int32_t *cnt = cnt_all + tid;
        const uint4 w = philox4x32_10(a.key0, a.key1, c0, s_tet[tid], 0u, (kPurposeReac << 28) | c3);
        const float neg_log_u1 = -steps_logf(unit24f(w.x));
        float a0 = 0.0f;
#pragma unroll
        for (int r = 0; r < RM; ++r) {
            if (r < m.R) {
                const float ar = ((active >> r) & 1u) ? propensity(m.reac[r], cnt, BLOCK, inv_nav) : 0.0f;
                a0 = __fadd_rn(a0, ar);
            }
        }
        if (a0 > 0.0f) {
            const float dt = __fdiv_rn(neg_log_u1, a0);
            if (!(dt > a.tau_dn)) {
                queue[atomicAdd(&nqueue, 1)] = tid;
                reacted[tid] = 1;
            }
        }
    }
    __syncthreads();

    // ---- C1 + B: the tets that did not react already have their trial counts
    // (their counts); their work items are grabbed by every warp while the
    // first warps run the full SSA of the tets that did (B), then join in.
    uint32_t W = (live && !reacted[tid]) ? trial_words(m, a, s_thr[tid], trial_all + tid, BLOCK) : 0u;
    words[tid] = W;
    uint32_t total = block_exclusive_scan<BLOCK>((W + kItemWords - 1u) / kItemWords, blk_start, warp_tot);
    if (tid == 0) {
        blk_start[BLOCK] = total;
        next_item = 0;
    }
    map_items<BLOCK>(tid, W, blk_start[tid], total, trial_all + tid, item_owner, item_before);
    __syncthreads();
    const int nq = nqueue;
    if (tid < nq) {
        const int t = queue[tid];
        bad |= ssa_tet<BLOCK, RM>(m, a, cnt_all + t, trial_all + t, s_tet[t], c0, c3, s_inv_nav[t], s_mask[t]);
    }
    __syncwarp();
    {
        const int lane = tid & 31;
        for (;;) {
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(&next_item, 32u);
            base = __shfl_sync(0xFFFFFFFFu, base, 0);
            if (base >= total) break;
            const uint32_t item = base + (uint32_t)lane;
            if (item < total)
                diffuse_item<BLOCK>(a, item, total, nlive, blk_start, item_owner, item_before, words, trial_all,
                                    cnt_all, s_thr, s_nbr, s_tet, c0, c3);
        }
    }
    __syncthreads();
    // ---- C2: the work items of the tets that reacted, now that their trial counts are known
    W = (live && reacted[tid]) ? trial_words(m, a, s_thr[tid], trial_all + tid, BLOCK) : 0u;
    words[tid] = W;
    total = block_exclusive_scan<BLOCK>((W + kItemWords - 1u) / kItemWords, blk_start, warp_tot);
    if (tid == 0) blk_start[BLOCK] = total;
    map_items<BLOCK>(tid, W, blk_start[tid], total, trial_all + tid, item_owner, item_before);
    __syncthreads();
    for (uint32_t item = tid; item < total; item += BLOCK)
        diffuse_item<BLOCK>(a, item, total, nlive, blk_start, item_owner, item_before, words, trial_all, cnt_all,
                            s_thr, s_nbr, s_tet, c0, c3);
    __syncthreads();

    // ---- D: the molecules that stay (immobile species: written by this tet alone)
    if (live) {
        for (int s = 0; s < S; ++s) {
            const int32_t N = cnt_all[s * BLOCK + tid];
            int32_t *out = a.nxt + s * Tpad + i;
            if ((m.diffusive >> s) & 1u) {
                if (N) atomicAdd(out, N);
            } else {
                *out = N;
            }
        }
    }
    if (bad) atomicOr(a.err, bad);
}

}  // namespace
}  // namespace steps
