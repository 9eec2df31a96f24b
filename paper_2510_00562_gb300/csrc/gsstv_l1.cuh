// Exact threshold of the l1-ball projection (Sec. III-B) on the GPU.
//
// For x in R^n and radius r > 0 with ||x||_1 > r, the projection onto
// B_{1,r} is sign(x) max(|x| - tau, 0) where tau > 0 is the root of
//   phi(tau) = sum_i max(|x_i| - tau, 0) - r,
// a continuous, piecewise-linear, non-increasing function of tau.  Two ways
// to get tau, both exact up to floating-point rounding of the sums:
//
//  * window: given counts and sums of the |x| above a window (lo, hi] and the
//    values inside it (the candidates), Michelot's fixed point
//    tau <- (sum_{|x| > tau} |x| - r) / #{|x| > tau}, started from "every
//    candidate active", reaches the root in a few passes over the candidates.
//  * radix: for |x| >= 0 the IEEE bit pattern is monotone in the value, so a
//    histogram of the top 11 bits with per-bin counts and integer sums of the
//    remaining mantissa bits gives phi at every bin edge exactly; the bin that
//    brackets the root is refined on the next 11 and then 9 bits, after which
//    a bin holds a single value and the root follows in closed form.  Any
//    bracket small enough is finished by gathering it and running the window
//    step on it.
#pragma once

#include "gsstv_internal.cuh"

namespace gsstv {

// What a window pass learned besides tau (for placing a retry window).
struct WinInfo {
    double phi_hi = 0.0;   // phi at the top of the window
    double phi_lo = 0.0;   // phi at the bottom (valid when the candidates fit)
    double n_lo = 0.0;     // count of |x| > theta_lo
};

// Calls f(x, k) for every candidate x = cand[k], k < m, with kCandBatch
// 16-byte loads in flight per thread (then four, then one): one CTA walking a
// long candidate list is bound by the latency of its loads, not by their
// bandwidth.  cand must be 16-byte aligned (every candidate buffer starts on
// a 256-byte boundary).
constexpr int kCandBatch = 4;
template <int B, typename F>
__device__ __forceinline__ unsigned candidate_batches(const float4* c4, unsigned k, unsigned m4, unsigned nt, F& f) {
    for (; k + (B - 1u) * nt < m4; k += B * nt) {
        float4 q[B];
#pragma unroll
        for (int j = 0; j < B; ++j) q[j] = __ldcg(c4 + k + j * nt);
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const unsigned b = 4u * (k + j * nt);
            f(q[j].x, b); f(q[j].y, b + 1u); f(q[j].z, b + 2u); f(q[j].w, b + 3u);
        }
    }
    return k;
}
template <typename F>
__device__ __forceinline__ void for_each_candidate(const float* cand, unsigned m, F&& f) {
    const unsigned nt = blockDim.x, m4 = m / 4u;
    const float4* c4 = reinterpret_cast<const float4*>(cand);
    unsigned k = threadIdx.x;
    k = candidate_batches<kCandBatch>(c4, k, m4, nt, f);
    if (kCandBatch > 4) k = candidate_batches<4>(c4, k, m4, nt, f);
    for (; k < m4; k += nt) {
        const float4 q = __ldcg(c4 + k);
        f(q.x, 4u * k); f(q.y, 4u * k + 1u); f(q.z, 4u * k + 2u); f(q.w, 4u * k + 3u);
    }
    for (unsigned j = 4u * m4 + threadIdx.x; j < m; j += nt) f(__ldcg(cand + j), j);
}

// Many candidates: before Michelot's step, narrow the window on the GPU's
// float keys.  For x >= 0 the IEEE bit pattern is monotone in the value;
// bins of 2^shift keys aligned to multiples of 2^shift (shift <= 20) never
// straddle an exponent, so the sum of a bin's values is exact:
//   count x (value of the bin's lowest key) + ulp x (sum of key residues).
// One pass over the candidates fills at most kNarrowBins bins; phi at every
// bin edge follows, and the bin whose lower edge is the highest with
// phi >= 0 brackets the root; the bins above it join the "above" count and
// sum.  Repeated on that bin until it holds at most kNarrowStage values,
// which are then staged in the scratch for Michelot's step.
constexpr unsigned kNarrowStage = 3 * kNarrowBins;   // floats the scratch stages
constexpr unsigned kNarrowMin = 4096;                // candidates beyond this are narrowed first
constexpr unsigned kWarpMichelot = 1024;             // narrowed values this few: one warp finishes

// Bin geometry of one narrowing round over the key window (klo, khi]: bins of
// 2^shift keys counted from base = klo >> shift, nb of them, with the
// smallest shift that needs at most kNarrowBins bins.  ok: the window spans
// at most 16 binary orders (then nb <= kNarrowBins and the integer sums of
// the bins are exact).
struct NarrowGeom {
    unsigned base;
    int shift, nb;
    bool ok;
};
__device__ __forceinline__ NarrowGeom narrow_geom(unsigned klo, unsigned khi) {
    NarrowGeom g;
    g.shift = 0;
    while (g.shift < 20 && ((khi >> g.shift) - (klo >> g.shift)) >= (unsigned)kNarrowBins) ++g.shift;
    g.base = klo >> g.shift;
    g.nb = (int)((khi >> g.shift) - g.base) + 1;
    g.ok = max((int)((khi >> 23) & 0xffu), 1) - max((int)(((klo + 1u) >> 23) & 0xffu), 1) <= 16;
    return g;
}
// A narrowing histogram is kNarrowBins 64-bit words (8-byte aligned, shared
// or global memory), bin b holding its count in the bits from kNarrowCntBit
// up and the sum of its keys' residues below the bin edge in the bits below:
// a residue is below 2^20 (shift <= 20), and a histogram that is read holds at
// most kCandCap = 2^20 keys, so the sum stays below 2^40 and the count below
// 2^22.  One 64-bit atomic counts a key.
constexpr int kNarrowCntBit = 42;
__device__ __forceinline__ void narrow_add(unsigned* h, const NarrowGeom& g, unsigned key) {
    const int b = (int)((key >> g.shift) - g.base);
    const unsigned res = key - ((key >> g.shift) << g.shift);
    atomicAdd(reinterpret_cast<unsigned long long*>(h) + b, (1ull << kNarrowCntBit) + res);
}
__device__ __forceinline__ unsigned narrow_count(unsigned long long w) { return (unsigned)(w >> kNarrowCntBit); }
__device__ __forceinline__ unsigned long long narrow_res(unsigned long long w) {
    return w & ((1ull << kNarrowCntBit) - 1ull);
}
// The key histogram of vector v's candidate list when every one of its m
// candidates was counted into it (built by the passes that appended them,
// over the same window), else null.
__device__ __forceinline__ const unsigned* narrow_pre(const L1Work& w, int v, unsigned m) {
    return (w.nh && m > 0u && __ldcg(w.nbinned + v) == m) ? w.nh + v * 3 * kNarrowBins : nullptr;
}
// Clears vector v's list histogram after its finish has read it (whole block).
__device__ __forceinline__ void narrow_clear(const L1Work& w, int v) {
    if (!w.nh) return;
    const unsigned used = __ldcg(w.nbinned + v);
    __syncthreads();
    if (used == 0u) return;
    for (int k = threadIdx.x; k < 2 * kNarrowBins; k += blockDim.x) w.nh[v * 3 * kNarrowBins + k] = 0u;
    if (threadIdx.x == 0) w.nbinned[v] = 0u;
}

// Whole block.  cand[0..m): the candidates, every one in (klo, khi] as keys;
// scr: 3 kNarrowBins unsigned of shared memory; sh_d: 4 doubles of shared
// memory; pre (optional): the candidates' key
// histogram over (klo, khi], already built (the first round reads it instead
// of binning the candidates).  On
// return 0: (klo, khi] narrowed, n_hi / s_hi now count everything above khi,
// and the *m_st values in the new window are staged as floats in scr.
// Returns 1 when phi at the window's lower end is negative (the root lies
// below it; sh_d[2], sh_d[3]: phi there and the count above it), 2 when the
// window is too wide to narrow (more than 16 binary orders) or does not
// narrow in a few rounds.
static __device__ int l1_narrow(const float* cand, bool cand_shared, unsigned m, double& n_hi, double& s_hi,
                                unsigned& klo, unsigned& khi, double r, unsigned* scr, unsigned* m_st, int* sh_i,
                                double* sh_d, const unsigned* pre = nullptr) {
    // every candidate, from global memory (batched loads) or from shared memory
    auto each = [&](auto&& f) {
        if (cand_shared) {
            for (unsigned k = threadIdx.x; k < m; k += blockDim.x) f(cand[k], k);
        } else {
            for_each_candidate(cand, m, f);
        }
    };
    const unsigned long long* hw = reinterpret_cast<const unsigned long long*>(scr);
    for (int round = 0; round < 8; ++round) {
        const NarrowGeom ng = narrow_geom(klo, khi);
        const int shift = ng.shift;
        const unsigned base = ng.base;
        const int nb = ng.nb;
        // the integer sums below need a window of at most 16 binary orders
        if (!ng.ok) return 2;
        __syncthreads();
        if (round == 0 && pre) {
            // 16-byte loads, all of a thread's issued before its stores (one
            // CTA copying from L2 is bound by the loads' latency)
            const uint4* p4 = reinterpret_cast<const uint4*>(pre);
            uint4* s4 = reinterpret_cast<uint4*>(scr);
            constexpr int kW4 = 2 * kNarrowBins / 4;
            uint4 q[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int k = (int)threadIdx.x + j * (int)blockDim.x;
                if (k < kW4) q[j] = __ldcg(p4 + k);
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int k = (int)threadIdx.x + j * (int)blockDim.x;
                if (k < kW4) s4[k] = q[j];
            }
            for (int k = (int)threadIdx.x + 2 * (int)blockDim.x; k < kW4; k += blockDim.x) s4[k] = __ldcg(p4 + k);
        } else {
            for (int k = threadIdx.x; k < 2 * kNarrowBins; k += blockDim.x) scr[k] = 0u;
            __syncthreads();
            each([&](float x, unsigned) {
                const unsigned key = __float_as_uint(x);
                if (key > klo && key <= khi) narrow_add(scr, ng, key);
            });
        }
        __syncthreads();
        // Exact sums in units of u0, the ulp at the window's lowest key: every
        // float in the window is an integer multiple of u0 (below 2^40 of
        // them while the window spans at most 16 binary orders), so a bin's
        // count and sum and their suffix sums are exact 64-bit integers, and
        // the sign of phi at a bin edge follows from an integer comparison.
        const unsigned k0 = klo + 1u;
        const int e0 = max((int)((k0 >> 23) & 0xffu), 1);
        const double u0 = key_ulp(k0);
        auto V = [&](unsigned key) -> unsigned long long {       // value / u0 of a key in the window
            const unsigned e = (key >> 23) & 0xffu;
            const unsigned long long mant = (key & 0x7fffffu) | (e ? 0x800000u : 0u);
            return mant << (max((int)e, 1) - e0);
        };
        auto bin_int = [&](int b) -> unsigned long long {        // sum of bin b, in units of u0
            const unsigned lk = (base + (unsigned)b) << shift;
            const unsigned long long w = hw[b];
            return (unsigned long long)narrow_count(w) * V(lk) + (narrow_res(w) << (max((int)((lk >> 23) & 0xffu), 1) - e0));
        };
        // phi at an edge with the bins from b up and everything above the window
        auto phi_at = [&](double e, unsigned long long e_int, unsigned long long Nsuf, unsigned long long Ssuf) {
            return s_hi - n_hi * e - r + (double)(long long)(Ssuf - Nsuf * e_int) * u0;
        };
        auto edge_phi = [&](int b, unsigned long long Nsuf, unsigned long long Ssuf) {
            if (b == 0)       // the window's lower end (exclusive)
                return s_hi + (double)Ssuf * u0 - (n_hi + (double)Nsuf) * (double)__uint_as_float(klo) - r;
            const unsigned lk = (base + (unsigned)b) << shift;
            return phi_at((double)__uint_as_float(lk), V(lk), Nsuf, Ssuf);
        };
        // The bin whose lower edge is the highest with phi >= 0 (phi does not
        // increase with the edge, so those edges come first).  Warp 0 alone:
        // FP64 runs at a small fraction of the FP32 rate on this part, and one
        // warp's FP64 instruction costs what the whole block's would divided
        // by its warps.  Each lane sums a chunk of at most 64 bins; the
        // highest lane whose chunk's lowest edge has phi >= 0 holds the bin,
        // which the lanes then find two bins each.
        if (threadIdx.x < 32) {
            const int lane = (int)threadIdx.x;
            // phi at an edge e inside the window (b > 0) is A + u0 X with
            // A = s_hi - r and the exact integer X = Ssuf - (Nsuf + n_hi) e/u0,
            // so phi >= 0 exactly when X >= T = ceil(-A / u0) (u0 a power of
            // two: the quotient is exact): the lanes test in integers, lane 0
            // alone computes T in FP64.  Windows so narrow against the sums
            // that T leaves 62 bits take the FP64 test.
            long long T = 0, NH = 0;
            int int_ok = 0;
            if (lane == 0) {
                const double q = ceil(-(s_hi - r) / u0);
                int_ok = fabs(q) < 4.6e18 && n_hi >= 0.0 && n_hi < 9.0e15;
                T = int_ok ? (long long)q : 0;
                NH = int_ok ? (long long)n_hi : 0;
            }
            int_ok = __shfl_sync(0xffffffffu, int_ok, 0);
            T = __shfl_sync(0xffffffffu, T, 0);
            NH = __shfl_sync(0xffffffffu, NH, 0);
            auto edge_ok = [&](int b, unsigned long long Nsuf, unsigned long long Ssuf) -> bool {
                if (b == 0 || !int_ok) return edge_phi(b, Nsuf, Ssuf) >= 0.0;
                const unsigned lk = (base + (unsigned)b) << shift;
                const __int128 X = (__int128)Ssuf - (__int128)(Nsuf + (unsigned long long)NH) * (__int128)V(lk);
                return X >= (__int128)T;
            };
            const int per = (nb + 31) / 32;
            const int c0 = lane * per, c1 = min(nb, c0 + per);
            unsigned long long Nc = 0, Sc = 0;
            for (int b = c0; b < c1; ++b) { Nc += narrow_count(hw[b]); Sc += bin_int(b); }
            // inclusive suffix over the lanes: the bins from c0 up
            unsigned long long Ni = Nc, Si = Sc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long x = __shfl_down_sync(0xffffffffu, Ni, o);
                const unsigned long long y = __shfl_down_sync(0xffffffffu, Si, o);
                if (lane + o < 32) { Ni += x; Si += y; }
            }
            const bool ok = c0 < c1 && edge_ok(c0, Ni, Si);
            const unsigned okm = __ballot_sync(0xffffffffu, ok);
            if (okm == 0u) {
                if (lane == 0) {
                    sh_i[0] = -1;
                    // phi at the window's lower end, and the count above it
                    sh_d[2] = edge_phi(0, Ni, Si);
                    sh_d[3] = n_hi + (double)Ni;
                }
            } else {
                const int L = 31 - __clz(okm);
                const int l0 = L * per, l1 = min(nb, l0 + per);
                // the bins above lane L's chunk
                const unsigned long long Nup = __shfl_sync(0xffffffffu, Ni - Nc, L);
                const unsigned long long Sup = __shfl_sync(0xffffffffu, Si - Sc, L);
                const int bA = l0 + 2 * lane, bB = bA + 1;
                const unsigned long long nA = bA < l1 ? narrow_count(hw[bA]) : 0ull, sA = bA < l1 ? bin_int(bA) : 0ull;
                const unsigned long long nB = bB < l1 ? narrow_count(hw[bB]) : 0ull, sB = bB < l1 ? bin_int(bB) : 0ull;
                unsigned long long Nj = nA + nB, Sj = sA + sB;      // inclusive suffix from bA
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned long long x = __shfl_down_sync(0xffffffffu, Nj, o);
                    const unsigned long long y = __shfl_down_sync(0xffffffffu, Sj, o);
                    if (lane + o < 32) { Nj += x; Sj += y; }
                }
                const bool okA = bA < l1 && edge_ok(bA, Nup + Nj, Sup + Sj);
                const bool okB = bB < l1 && edge_ok(bB, Nup + Nj - nA, Sup + Sj - sA);
                const int mine = okB ? bB : okA ? bA : -1;
                const int best = __reduce_max_sync(0xffffffffu, mine);
                if (mine == best) {
                    // the bins above the chosen one
                    const unsigned long long an = best == bB ? Nup + Nj - nA - nB : Nup + Nj - nA;
                    const unsigned long long as = best == bB ? Sup + Sj - sA - sB : Sup + Sj - sA;
                    sh_i[0] = best;
                    sh_d[0] = n_hi + (double)an;
                    sh_d[1] = s_hi + (double)as * u0;
                }
            }
        }
        __syncthreads();
        const int kb = sh_i[0];
        if (kb < 0) { __syncthreads(); return 1; }
        const unsigned count = narrow_count(hw[kb]);
        n_hi = sh_d[0];
        s_hi = sh_d[1];
        const unsigned nlo = kb == 0 ? klo : ((base + (unsigned)kb) << shift) - 1u;
        const unsigned nhi = min(khi, ((base + (unsigned)kb + 1u) << shift) - 1u);
        klo = nlo;
        khi = nhi;
        __syncthreads();
        if (count <= kNarrowStage) {
            // stage the bracket bin's values
            if (threadIdx.x == 0) sh_i[0] = 0;
            __syncthreads();
            float* st = reinterpret_cast<float*>(scr);
            each([&](float x, unsigned) {
                const unsigned key = __float_as_uint(x);
                if (key > klo && key <= khi) st[atomicAdd(sh_i, 1)] = x;
            });
            __syncthreads();
            *m_st = (unsigned)sh_i[0];
            __syncthreads();
            return 0;
        }
    }
    return 2;   // did not narrow enough (only float keys closer than 2^-20 relative could do this)
}

// Michelot's fixed point restricted to a window.  One whole block calls it.
// n_hi, s_hi: count and sum of |x| > theta_hi; cand[0..m_raw): every |x| in
// (theta_lo, theta_hi].  Returns 0 with *tau_out; 2 when the root lies above
// the window; 1 when it lies below or the candidates overflowed the buffer.
// stage (optional): shared memory for stage_cap floats that the block no
// longer uses; when the candidates fit they are copied there on the first
// pass and every later pass reads them from it instead of from L2.
// scr (optional): 3 kNarrowBins unsigned of shared memory; with more than
// kNarrowMin candidates the window is first narrowed on the float keys
// (l1_narrow; from the stage when they fit it, else from global memory), so
// that Michelot's passes run over the few values of one narrow bin instead
// of every candidate.  pre (optional): the candidates' key histogram over the
// window, built while they were appended; the first narrowing round then
// reads it, and only the values of the chosen bin are staged (one pass over
// the list).
static __device__ int l1_window_finish(double n_hi, double s_hi, const float* cand, unsigned m_raw,
                                       double theta_lo, double theta_hi, double r,
                                       double* tau_out, double* red_d,
                                       unsigned long long* red_u, WinInfo* info = nullptr,
                                       float* stage = nullptr, unsigned stage_cap = 0,
                                       unsigned* scr = nullptr, const unsigned* pre = nullptr) {
    // The scalar tests in FP64 on thread 0 (FP64 is scarce on this part),
    // shared with the block.
    __shared__ int wp_rc, wp_narrow, wp_pre;
    __shared__ unsigned wp_klo, wp_khi;
    if (threadIdx.x == 0) {
        const double phi_hi = s_hi - n_hi * theta_hi - r;
        if (info) info->phi_hi = phi_hi;
        wp_rc = m_raw > kCandCap ? 1 : phi_hi > 0.0 ? 2 : -1;     // 2: root above the window
        wp_narrow = wp_rc < 0 && scr && m_raw > kNarrowMin && theta_lo >= 0.0;
        // the window's ends as float keys: (klo, khi] holds every candidate
        unsigned klo = __float_as_uint((float)theta_lo), khi = __float_as_uint((float)theta_hi);
        if ((double)__uint_as_float(klo) > theta_lo) klo -= 1u;        // rounding of the ends
        if ((double)__uint_as_float(khi) < theta_hi) khi += 1u;
        wp_klo = klo;
        wp_khi = khi;
        // a key histogram built over the float window fits only that window
        wp_pre = pre && (double)(float)theta_lo == theta_lo && (double)(float)theta_hi == theta_hi;
    }
    __syncthreads();
    if (wp_rc >= 0) {
        const int rc = wp_rc;
        __syncthreads();
        return rc;
    }
    unsigned m = m_raw;
    if (wp_narrow) {
        unsigned klo = wp_klo, khi = wp_khi;
        if (!wp_pre) pre = nullptr;
        unsigned m_st = 0;
        __shared__ int nr_i[1];
        double nh = n_hi, sh = s_hi;
        // with a stage that holds them, the candidates are read from global
        // memory once and narrowed from shared memory
        const float* src = cand;
        bool src_shared = false;
        if (stage && m <= stage_cap && !pre) {
            for_each_candidate(cand, m, [&](float x, unsigned k) { stage[k] = x; });
            __syncthreads();
            src = stage;
            src_shared = true;
        }
        // (red_d serves as the narrowing's scalars)
        const int rc = l1_narrow(src, src_shared, m, nh, sh, klo, khi, r, scr, &m_st, nr_i, red_d, pre);
        if (rc == 1) {
            // phi(theta_lo) < 0: as below, inside the ball or a miss below
            if (info) { info->phi_lo = red_d[2]; info->n_lo = red_d[3]; }
            if (theta_lo <= 0.0) { *tau_out = 0.0; return 0; }
            return 1;
        }
        if (rc == 0) {
            // Michelot on the staged values of the bracket bin
            n_hi = nh;
            s_hi = sh;
            cand = nullptr;
            stage = reinterpret_cast<float*>(scr);
            stage_cap = kNarrowStage;
            m = m_st;
            theta_lo = (double)__uint_as_float(klo);
            theta_hi = (double)__uint_as_float(khi);
            if (info) info = nullptr;                  // the window's own phi_lo is not computed here
        }
    }
    const bool staged = stage && m <= stage_cap;
    const bool pre_staged = cand == nullptr;           // the narrowed values already sit in the stage
    if ((pre_staged || staged) && m <= kWarpMichelot) {
        // A few values (one narrow bin, or a small window): warp 0 alone runs
        // Michelot's steps on them, with shuffles instead of CTA barriers;
        // the FP64 steps on lane 0.
        __shared__ double ww_tau;
        __shared__ int ww_rc;
        if (!pre_staged) {
            for (unsigned k = threadIdx.x; k < m; k += blockDim.x) stage[k] = __ldcg(cand + k);
            __syncthreads();
        }
        if (threadIdx.x < 32) {
            const unsigned lane = threadIdx.x;
            Kahan ks;
            for (unsigned k = lane; k < m; k += 32u) ks.add(stage[k]);
            float h, l;
            warp_sum_pair(ks, h, l);
            int state = 0;
            double tau = 0.0;
            float tf = 0.f;
            if (lane == 0) {
                const double sum_c = (double)h + (double)l;
                const double n_all = n_hi + (double)m;
                const double phi_lo = s_hi + sum_c - n_all * theta_lo - r;
                if (info) { info->phi_lo = phi_lo; info->n_lo = n_all; }   // (thread 0's)
                if (phi_lo < 0.0) {
                    state = theta_lo <= 0.0 ? 2 : 3;
                } else {
                    tau = (s_hi + sum_c - r) / n_all;
                    tf = __double2float_rd(tau);
                }
            }
            state = __shfl_sync(0xffffffffu, state, 0);
            tf = __shfl_sync(0xffffffffu, tf, 0);
            int rc = state == 2 ? 0 : state == 3 ? 1 : 0;
            if (state == 0) {
                unsigned prev = m;
                for (int it = 0; it < 200; ++it) {
                    Kahan ka;
                    unsigned c = 0;
                    for (unsigned k = lane; k < m; k += 32u) {
                        const float x = stage[k];
                        if (x > tf) { ka.add(x); ++c; }
                    }
                    warp_sum_pair(ka, h, l);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
                    int done = 0;
                    if (lane == 0) {
                        tau = (s_hi + ((double)h + (double)l) - r) / (n_hi + (double)c);
                        tf = __double2float_rd(tau);
                        done = c == prev ? 1 : 0;
                    }
                    tf = __shfl_sync(0xffffffffu, tf, 0);
                    done = __shfl_sync(0xffffffffu, done, 0);
                    prev = c;
                    if (done) break;
                }
            }
            if (lane == 0) {
                ww_tau = state == 2 ? 0.0 : tau;
                ww_rc = rc;
            }
        }
        __syncthreads();
        const int rc = ww_rc;
        if (rc == 0) *tau_out = ww_tau;
        __syncthreads();
        return rc;
    }
    // Sums in compensated FP32 per thread and float pairs across the CTA;
    // the FP64 steps (a handful per pass) run on thread 0 and reach the
    // other threads through shared memory.
    __shared__ float2 wf_pair[32];
    __shared__ double wf_tau;
    __shared__ float wf_tf;
    __shared__ int wf_state;                          // 0 continue, 1 done, 2 inside, 3 below
    Kahan ks;
    if (pre_staged) {
        for (unsigned k = threadIdx.x; k < m; k += blockDim.x) ks.add(stage[k]);
    } else {
        for_each_candidate(cand, m, [&](float x, unsigned k) {
            if (staged) stage[k] = x;
            ks.add(x);
        });
    }
    const double sum_c = block_sum_pair(ks, wf_pair);       // (its barriers publish the stage)
    if (threadIdx.x == 0) {
        const double n_all = n_hi + (double)m;
        const double phi_lo = s_hi + sum_c - n_all * theta_lo - r;
        if (info) { info->phi_lo = phi_lo; info->n_lo = n_all; }
        if (phi_lo < 0.0) {
            wf_state = theta_lo <= 0.0 ? 2 : 3;
        } else {
            wf_state = 0;
            wf_tau = (s_hi + sum_c - r) / n_all;
            wf_tf = __double2float_rd(wf_tau);
        }
    }
    __syncthreads();
    const int st0 = wf_state;
    if (st0 == 2) { *tau_out = 0.0; __syncthreads(); return 0; }   // inside the ball
    if (st0 == 3) { __syncthreads(); return 1; }                    // root below the window
    unsigned long long prev = m;
    for (int it = 0; it < 200; ++it) {
        // for a float x, x > tau exactly when x > (tau rounded down to float):
        // the test runs in FP32
        const float tf = wf_tf;
        Kahan ka;
        unsigned c = 0;
        auto take = [&](float x, unsigned) { if (x > tf) { ka.add(x); ++c; } };
        if (staged) {
            for (unsigned k = threadIdx.x; k < m; k += blockDim.x) take(stage[k], k);
        } else {
            for_each_candidate(cand, m, take);
        }
        const double sa = block_sum_pair(ka, wf_pair);
        const unsigned long long ca = block_count(c, red_u);
        if (threadIdx.x == 0) {
            wf_tau = (s_hi + sa - r) / (n_hi + (double)ca);
            wf_tf = __double2float_rd(wf_tau);
            wf_state = ca == prev ? 1 : 0;
        }
        __syncthreads();
        const bool done = wf_state == 1;
        prev = ca;
        if (done) break;
    }
    *tau_out = wf_tau;
    __syncthreads();
    return 0;
}

// After a missed window: place one retry window from the bounds the miss
// gives, or fall back to the radix search.  phi is convex, non-increasing,
// with slope -#{|x| > tau}, so
//   root above (phi(hi) > 0):  tau >= hi + phi(hi) / n_hi          (lower bound)
//   root below (phi(lo) < 0):  tau <= lo + phi(lo) / n(lo)         (upper bound)
// The retry window extends from the bound away from the old window by four
// times the distance, capped near kRetryTarget expected candidates (wider than
// K1's windows: one retry pass costs far less than the radix passes a second
// miss leads to).  Thread 0 only.
static __device__ void l1_after_miss(L1Ctl& c, int rc, const WinInfo& wi, double n_hi, unsigned m,
                                     double lo, double hi) {
    // A retry needs a density estimate, and its capped width must cover at
    // least half the jump the bound implies; otherwise it would most likely
    // miss again and the radix passes run at once.
    double a = -1.0, b = -1.0;
    if (rc == 2 && n_hi > 0.0 && c.dens > 0.0) {
        const double lb = hi + wi.phi_hi / n_hi;
        const double w = fmin(fmax(4.0 * (lb - hi), 1e-6 * lb), kRetryTarget / c.dens);
        if (w >= 0.5 * (lb - hi)) {
            a = lb;
            b = lb + w;
        }
    } else if (rc == 1 && m <= kCandCap && wi.n_lo > 0.0 && lo > 0.0 && c.dens > 0.0) {
        const double ub = lo + wi.phi_lo / wi.n_lo;
        const double w = fmin(fmax(4.0 * (lo - ub), 1e-6 * lo), kRetryTarget / c.dens);
        if (w >= 0.5 * (lo - ub)) {
            a = fmax(ub - w, 0.0);
            b = ub;
        }
    }
    c.prefix = 0; c.n_above = 0; c.s_above = 0.0;
    c.hist_left = kHistPasses;
    if (b > a && a >= 0.0) {
        c.need = NEED_WINDOW;
        c.g_lo = __double2float_rd(a);
        c.g_hi = __double2float_ru(b);
    } else {
        c.need = NEED_RADIX0;
        c.exact_runs++;
    }
}

// Value of the lower edge of histogram bin b (b = kK1Bins: the top edge).
__device__ __forceinline__ float hist_edge(unsigned hbase, int b) {
    return __uint_as_float((hbase + (unsigned)b) << kHistShift);
}
// Is a histogram based at hbase made of finite, positive bin edges?
__host__ __device__ __forceinline__ bool hist_base_ok(unsigned hbase) {
    return hbase > 0u && ((unsigned long long)(hbase + kK1Bins) << kHistShift) < 0x7f800000ull;
}

// After K1's window missed: a bracket of the root estimated from K1's sampled
// histogram of |x|.  hist_g: kK1Bins counts of a 1/scale sample (global; hist:
// kK1Bins unsigned of shared memory to read them into), bin b holding
// the sampled |x| in [e_b, e_{b+1}) with e_b = hist_edge(hbase, b); n_top,
// s_top: count and sum of the sampled |x| >= e_top.  Scaled up, and with every
// binned value taken at its bin's lower (upper) edge, they estimate phi at each
// edge from below (above); the highest edge whose lower estimate is >= 0 and
// the lowest edge above it whose upper estimate is < 0 bracket the root, and
// the bracket is widened by two bins on each side for the sampling error.
// Returns 1 with the window (*lo, *hi] and the expected number of values
// inside it in *m, or 0 when the range does not bracket the root or the
// window would hold more than half of kCandCap values.  The retry pass on the
// window computes everything exactly (a wrong bracket costs only time).  One
// whole block calls it; warp 0 works.
static __device__ int l1_hist_bracket(const unsigned* hist_g, unsigned hbase, double n_top, double s_top,
                                      double r, double scale, float* lo_out, float* hi_out, double* m_out,
                                      int* sh_i, unsigned* hist) {
    constexpr int PER = kK1Bins / 32;
    constexpr int WIDEN = 2;
    // the counts into shared memory (every thread, loads in parallel)
    __syncthreads();
    for (int k = threadIdx.x; k < kK1Bins; k += blockDim.x) hist[k] = __ldcg(hist_g + k);
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const int b0 = lane * PER;
        // estimates from a sample: FP32 arithmetic is precise enough
        const float fs = (float)scale;
        const float nt_ = (float)(n_top * scale), st_ = (float)(s_top * scale), rf = (float)r;
        float c_l = 0.f, sl_l = 0.f, sh_l = 0.f;
        for (int b = b0; b < b0 + PER; ++b) {
            const float c = fs * (float)hist[b];
            c_l += c;
            sl_l += c * hist_edge(hbase, b);
            sh_l += c * hist_edge(hbase, b + 1);
        }
        // totals of the lanes above this one (exclusive suffix)
        float c_in = c_l, sl_in = sl_l, sh_in = sh_l;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float c = __shfl_down_sync(0xffffffffu, c_in, o);
            const float a = __shfl_down_sync(0xffffffffu, sl_in, o);
            const float b = __shfl_down_sync(0xffffffffu, sh_in, o);
            if (lane + o < 32) { c_in += c; sl_in += a; sh_in += b; }
        }
        const float top = hist_edge(hbase, kK1Bins);
        const float phi_top = st_ - nt_ * top - rf;
        // pass 1: the highest edge whose lower estimate is >= 0
        float N = nt_ + (c_in - c_l), SL = st_ + (sl_in - sl_l);
        int a_best = phi_top >= 0.f ? kK1Bins : -1;
        for (int b = b0 + PER - 1; b >= b0 && a_best < 0; --b) {
            const float e = hist_edge(hbase, b);
            const float c = fs * (float)hist[b];
            N += c;
            SL += c * e;
            if (SL - N * e - rf >= 0.f) a_best = b;
        }
        int a_all = a_best;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a_all = max(a_all, __shfl_xor_sync(0xffffffffu, a_all, o));
        // pass 2: the lowest edge above it whose upper estimate is < 0
        int c_best = kK1Bins + 1;
        if (a_all >= 0 && a_all < kK1Bins) {
            if (phi_top < 0.f) c_best = kK1Bins;
            N = nt_ + (c_in - c_l);
            float SH = st_ + (sh_in - sh_l);
            for (int b = b0 + PER - 1; b >= b0; --b) {
                const float e = hist_edge(hbase, b);
                const float c = fs * (float)hist[b];
                N += c;
                SH += c * hist_edge(hbase, b + 1);
                if (b > a_all && SH - N * e - rf < 0.f) c_best = b;   // the lowest such b of this lane
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c_best = min(c_best, __shfl_xor_sync(0xffffffffu, c_best, o));
        const bool found = a_all >= 0 && a_all < kK1Bins && c_best <= kK1Bins;
        const int lo_b = max(a_all - WIDEN, 0), hi_b = min(c_best + WIDEN, kK1Bins);
        // expected values inside the widened bracket [e_lo, e_hi)
        float m = 0.f;
        if (found)
            for (int b = b0; b < b0 + PER; ++b)
                if (b >= lo_b && b < hi_b) m += fs * (float)hist[b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
        if (lane == 0) {
            const bool ok = found && m <= 0.5f * (float)kCandCap;
            sh_i[0] = ok ? 1 : 0;
            if (ok) {
                *lo_out = hist_edge(hbase, lo_b);
                *hi_out = hist_edge(hbase, hi_b);
                *m_out = m;
            }
        }
    }
    __syncthreads();
    return sh_i[0];
}

// Records tau of this iteration and places the window of the next one around
// the extrapolation of the last thresholds.  In the passes after a miss
// (K1's histogram on) the window spans the linear and the quadratic
// extrapolations; otherwise it is centred on the linear one, and after a window
// hit the half-width covers twice the last change of the step plus a tenth of
// the step (the extrapolation error of a smoothly converging sequence), after
// a miss twice the step itself.  Each is capped so that about kCandTarget
// (kCandTargetWide while the histogram is on) candidates are expected (density
// measured at the last window).  `hit`: tau came from K1's window.  Thread 0
// only.
static __device__ void l1_record_tau(L1Ctl& c, double tau_new, double m_used, double width_used, bool hit) {
    c.tau_prev2 = c.tau_prev;
    c.have_prev2 = c.have_prev;
    c.tau_prev = c.tau;
    c.have_prev = c.have_tau;
    c.tau = tau_new;
    c.have_tau = 1;
    c.need = NEED_NONE;
    if (width_used > 0.0 && m_used > 0.0) c.dens = m_used / width_used;
    if (!(tau_new > 0.0)) {            // ball inactive: window (0, 0]
        c.theta_lo = 0.f;
        c.theta_hi = 0.f;
        c.window_ok = 1;
        return;
    }
    const bool trend = c.have_prev && c.tau_prev > 0.0;
    const double d1 = trend ? tau_new - c.tau_prev : 0.0;
    double center = tau_new + d1;
    double hw;
    if (!trend) {
        hw = 1e-3 * tau_new;
    } else if (c.hist_left > 0 && c.have_prev2 && c.tau_prev2 > 0.0) {
        // the passes after a miss, while the thresholds move fast: the window
        // spans the linear and the quadratic extrapolations (tau + d1 and
        // tau + 2 d1 - d0) with a margin of half their distance and a tenth
        // of the step, after a retry or an exact search as after a hit
        const double d0 = c.tau_prev - c.tau_prev2;
        center = tau_new + d1 + 0.5 * (d1 - d0);
        hw = fabs(d1 - d0) + 0.1 * fabs(d1) + 1e-7 * tau_new;
    } else if (hit && c.have_prev2 && c.tau_prev2 > 0.0) {
        const double d0 = c.tau_prev - c.tau_prev2;
        hw = 2.0 * fabs(d1 - d0) + 0.1 * fabs(d1) + 1e-7 * tau_new;
    } else {
        hw = 2.0 * fabs(d1) + 1e-7 * tau_new;
    }
    // a wide window while the thresholds move fast (the passes after a miss,
    // with K1's histogram on), where a hit saves a retry pass; else a narrow
    // one, which K1 and the finish handle faster
    if (c.dens > 0.0) hw = fmin(hw, 0.5 * (c.hist_left > 0 ? kCandTargetWide : kCandTarget) / c.dens);
    // the histogram of the next pass: four octaves from a quarter of the
    // predicted threshold
    c.hbase = center > 0.0 ? (__float_as_uint(__double2float_rd(0.25 * center)) >> kHistShift) : 0u;
    const double lo = fmax(center - hw, 0.0);
    const double hi = center + hw;
    c.theta_lo = __double2float_rd(lo);
    c.theta_hi = __double2float_ru(hi);
    c.window_ok = 1;
}

// Radix level geometry: bin of a key and its residue (the bits below the bin).
struct RadixLevel {
    int level;
    __device__ __forceinline__ int nbins() const { return level == 2 ? 512 : 2048; }
    // does the key belong to the bracket fixed by the previous levels?
    __device__ __forceinline__ bool inside(unsigned key, unsigned prefix) const {
        return level == 0 ? true : level == 1 ? ((key >> 20) == prefix) : ((key >> 9) == prefix);
    }
    __device__ __forceinline__ int bin(unsigned key) const {
        return level == 0 ? (int)(key >> 20) : level == 1 ? (int)((key >> 9) & 2047u) : (int)(key & 511u);
    }
    __device__ __forceinline__ unsigned residue(unsigned key) const {
        return level == 0 ? (key & 0xfffffu) : level == 1 ? (key & 0x1ffu) : 0u;
    }
    __device__ __forceinline__ unsigned lo_key(unsigned prefix, int k) const {
        return level == 0 ? ((unsigned)k << 20)
             : level == 1 ? ((prefix << 20) | ((unsigned)k << 9))
                          : ((prefix << 9) | (unsigned)k);
    }
    __device__ __forceinline__ unsigned next_prefix(unsigned prefix, int k) const {
        return level == 0 ? (unsigned)k : ((prefix << 11) | (unsigned)k);
    }
};

// Bracket selection after a radix histogram pass.  One whole block calls it
// with the merged histogram (hcnt, hres: nbins entries) of one vector.
// Updates c: either tau is known (NEED_NONE), or the bracket bin is to be
// gathered (NEED_GATHER), or refined at the next level.
static __device__ void l1_radix_select(L1Ctl& c, RadixLevel lv, const unsigned long long* hcnt,
                                       const unsigned long long* hres, double r, double* sh_d,
                                       unsigned long long* sh_u, int* sh_i) {
    const int nb = lv.nbins();
    const int nt = blockDim.x;
    const int per = (nb + nt - 1) / nt;
    const int k0 = threadIdx.x * per;
    const int k1 = min(nb, k0 + per);
    // 1. chunk totals
    unsigned long long cnt = 0;
    double sum = 0.0;
    for (int k = k0; k < k1; ++k) {
        const unsigned long long ck = __ldcg(hcnt + k);
        if (ck) {
            const unsigned key = lv.lo_key(c.prefix, k);
            sum += (double)ck * key_value(key) + key_ulp(key) * (double)__ldcg(hres + k);
            cnt += ck;
        }
    }
    // sh_d[0..nt) chunk sums, sh_u[0..nt) chunk counts; suffixes by thread 0
    sh_d[threadIdx.x] = sum;
    sh_u[threadIdx.x] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = c.s_above;
        unsigned long long n = c.n_above;
        for (int t = nt - 1; t >= 0; --t) {     // exclusive suffix: bins above chunk t
            const double st = sh_d[t];
            const unsigned long long nt_ = sh_u[t];
            sh_d[t] = s;
            sh_u[t] = n;
            s += st;
            n += nt_;
        }
    }
    __syncthreads();
    // 2. inside the chunk, from the top bin down: phi(lo_k) >= 0 ?
    double s_run = sh_d[threadIdx.x];
    unsigned long long n_run = sh_u[threadIdx.x];
    int best = -1;
    double best_phi = 0.0, best_s_above = 0.0;
    unsigned long long best_n_above = 0, best_cnt = 0;
    for (int k = k1 - 1; k >= k0; --k) {
        const unsigned long long ck = __ldcg(hcnt + k);
        const unsigned key = lv.lo_key(c.prefix, k);
        const double lo = key_value(key);
        const double sk = ck ? (double)ck * lo + key_ulp(key) * (double)__ldcg(hres + k) : 0.0;
        const double s_ge = s_run + sk;
        const unsigned long long n_ge = n_run + ck;
        const double phi = s_ge - (double)n_ge * lo - r;
        if (phi >= 0.0) {
            best = k; best_phi = phi; best_s_above = s_run; best_n_above = n_run; best_cnt = ck;
            break;
        }
        s_run = s_ge;
        n_run = n_ge;
    }
    __syncthreads();
    // 3. the highest bracket over the block
    if (threadIdx.x == 0) sh_i[0] = -1;
    __syncthreads();
    atomicMax(sh_i, best);
    __syncthreads();
    const int kb = sh_i[0];
    if (best == kb && kb >= 0) {
        const unsigned key = lv.lo_key(c.prefix, kb);
        const double lo = key_value(key);
        if (best_phi == 0.0) {
            l1_record_tau(c, lo, 0.0, 0.0, false);
        } else if (lv.level == 2) {
            // the bracket bin holds one value, inactive for any tau above it
            l1_record_tau(c, (best_s_above - r) / (double)best_n_above, 0.0, 0.0, false);
        } else if (best_cnt <= (unsigned long long)kGatherMax) {
            c.need = NEED_GATHER;
            c.g_lo = __uint_as_float(key);
            c.g_hi = __uint_as_float(lv.lo_key(c.prefix, kb + 1) - 1u);
            c.n_above = best_n_above;
            c.s_above = best_s_above;
        } else {
            c.need = lv.level == 0 ? NEED_RADIX1 : NEED_RADIX2;
            c.prefix = lv.next_prefix(c.prefix, kb);
            c.n_above = best_n_above;
            c.s_above = best_s_above;
        }
    }
    if (threadIdx.x == 0 && kb < 0) {
        // phi(lower edge of the whole range) < 0: at level 0 the vector is
        // inside the ball; deeper, only rounding can get here.
        const double lo0 = lv.level == 0 ? 0.0 : key_value(lv.lo_key(c.prefix, 0));
        l1_record_tau(c, lo0, 0.0, 0.0, false);
    }
    __syncthreads();
}

}  // namespace gsstv
