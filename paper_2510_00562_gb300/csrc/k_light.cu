// K2 (the light pass of one P-PDS iteration), the exact radix search for the
// l1 thresholds, state conversion kernels and the standalone l1 projection.
//
// K2 finishes Algorithm 1 once the l1 thresholds tau_s, tau_t are known:
//   s+ = P_{B1,alpha}(s~) = soft(s~, tau_s),  t+ = soft(t~, tau_t),
//   s' = 2 s+ - s,  t' = 2 t+ - t,
//   y3+ = y3 + g3 D_v t'                                   (needs row i+1)
//   y4' = y4 + g4 (u' + s' + t'),  q = y4' - g4 v,
// and reduces ||q||^2: the l2-ball step of Algorithm 1 (Eq. 23 through
// Moreau's identity, Eq. 3) is y4+ = (1 - c) q with c = min(1, eps g4 / ||q||),
// which the next iteration applies when it reads q.  It also reduces the two
// norms of the stopping rule (Eq. 28).
#include <algorithm>
#include <cstdint>
#include <mutex>
#include <type_traits>

#include "gsstv_internal.cuh"
#include "gsstv_l1.cuh"

namespace gsstv {
namespace {

constexpr int NT = 256;
constexpr int K2_ROWS = 8;   // rows per thread strip in K2

template <typename T> struct Vec4;
template <> struct Vec4<float> {
    static __device__ __forceinline__ float4 ld(const float* p) { return *reinterpret_cast<const float4*>(p); }
    static __device__ __forceinline__ void st(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
};
template <> struct Vec4<__nv_bfloat16> {
    static __device__ __forceinline__ float4 ld(const __nv_bfloat16* p) {
        uint2 r = *reinterpret_cast<const uint2*>(p);
        float2 a = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&r.x));
        float2 b = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&r.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float4 v) {
        __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
        uint2 r;
        r.x = *reinterpret_cast<unsigned*>(&a);
        r.y = *reinterpret_cast<unsigned*>(&b);
        *reinterpret_cast<uint2*>(p) = r;
    }
};
template <> struct Vec4<__half> {
    static __device__ __forceinline__ float4 ld(const __half* p) {
        uint2 r = *reinterpret_cast<const uint2*>(p);
        float2 a = __half22float2(*reinterpret_cast<__half2*>(&r.x));
        float2 b = __half22float2(*reinterpret_cast<__half2*>(&r.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    static __device__ __forceinline__ void st(__half* p, float4 v) {
        __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
        uint2 r;
        r.x = *reinterpret_cast<unsigned*>(&a);
        r.y = *reinterpret_cast<unsigned*>(&b);
        *reinterpret_cast<uint2*>(p) = r;
    }
};
// four stores of a quad, stochastically rounded for 16-bit storage
template <typename T>
__device__ __forceinline__ void st4S(T* p, const float4& v, SRStream& sr) {
    if constexpr (std::is_same<T, float>::value) {
        *reinterpret_cast<float4*>(p) = v;
    } else {
        stS(p, v.x, sr); stS(p + 1, v.y, sr); stS(p + 2, v.z, sr); stS(p + 3, v.w, sr);
    }
}

__device__ __forceinline__ float comp(const float4& v, int k) {
    return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
}
__device__ __forceinline__ void set_comp(float4& v, int k, float x) {
    if (k == 0) v.x = x; else if (k == 1) v.y = x; else if (k == 2) v.z = x; else v.w = x;
}

// ---------------------------------------------------------------------------
// K2
// ---------------------------------------------------------------------------
template <typename T>
struct K2Args {
    Geom g;
    const T *u, *u_n, *s, *t, *y3, *q;
    const float* v;
    T *s_n, *t_n, *y3_n, *q_n;
    IterParams p;
    Scal* sc;
    double* part;       // 3 doubles per CTA
    SlabPart sp;        // the bands updated, and this launch's CTAs among the stage's
};

// The CTA `bid` of `nblk` that share one cube's K2 (a launch of its own, or
// the cube's share of a batch launch).
template <typename T>
__device__ __forceinline__ void k2_body(const K2Args<T>& a, const int bid, const int nblk) {
    __shared__ double red_d[64];
    __shared__ int is_last;
    const Geom g = a.g;
    const IterParams& P = a.p;
    const float cs = (float)(1.0 - a.sc->c[P.parity]);
    const float tau_s = (float)a.sc->ctl[0].tau;
    const float tau_t = (float)a.sc->ctl[1].tau;
    const unsigned it32 = (unsigned)a.sc->iter;       // seeds the 16-bit rounding streams
    const int quads = g.p2 / 4;
    const int strips = (g.n1 + K2_ROWS - 1) / K2_ROWS;
    const long long items = (long long)(a.sp.o1 - a.sp.o0) * strips * quads;
    Kahan aq, adu, au;
    for (long long it = bid * (long long)NT + threadIdx.x; it < items; it += (long long)nblk * NT) {
        const int qd = (int)(it % quads);
        const long long rest = it / quads;
        const int strip = (int)(rest % strips);
        const int b = a.sp.o0 + (int)(rest / strips);
        const int j = qd * 4;
        const int i_s = strip * K2_ROWS;
        const int i_own = min(i_s + K2_ROWS, g.n1);            // own rows [i_s, i_own)
        const int i_last = min(i_s + K2_ROWS, g.n1 - 1);       // plus one halo row if any
        float4 y3m = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i_s >= 1) y3m = Vec4<T>::ld(a.y3 + g.at(b, i_s - 1, j));
        float4 tprev = y3m, y3prev = y3m;
        for (int i = i_s; i <= i_last; ++i) {
            const long long o = g.at(b, i, j);
            const float4 s4 = Vec4<T>::ld(a.s + o), t4 = Vec4<T>::ld(a.t + o);
            const float4 y34 = Vec4<T>::ld(a.y3 + o), q4 = Vec4<T>::ld(a.q + o);
            const bool own = i < i_own;
            float4 u0 = make_float4(0, 0, 0, 0), u1 = u0, v4 = u0;
            if (own) {
                u0 = Vec4<T>::ld(a.u + o);
                u1 = Vec4<T>::ld(a.u_n + o);
                v4 = *reinterpret_cast<const float4*>(a.v + o);
            }
            float4 sp4, tp4, qn4, tb4, y3n4;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float y4 = __fmul_rn(cs, comp(q4, k));
                float xs, xt;
                s_t_tilde(comp(s4, k), comp(t4, k), comp(y34, k), comp(y3m, k), comp(q4, k), cs, i,
                          g.n1, P.gamma_s, P.gamma_t, xs, xt);
                const float sp = soft(xs, tau_s), tp = soft(xt, tau_t);
                const float sb = 2.f * sp - comp(s4, k), tb = 2.f * tp - comp(t4, k);
                set_comp(sp4, k, sp);
                set_comp(tp4, k, tp);
                set_comp(tb4, k, tb);
                // y3 of the row above, now that t' of this row is known
                set_comp(y3n4, k, comp(y3prev, k) + P.gamma_y3 * (tb - comp(tprev, k)));
                if (own) {
                    const float uo = comp(u0, k), un = comp(u1, k);
                    const float ub = 2.f * un - uo;
                    const float y4p = y4 + P.gamma_y4 * (ub + sb + tb);
                    const float qn = y4p - P.gamma_y4 * comp(v4, k);
                    set_comp(qn4, k, qn);
                    if (j + k < g.n2) {
                        aq.add(qn * qn);
                        const float du = un - uo;
                        adu.add(du * du);
                        au.add(uo * uo);
                    }
                }
            }
            SRStream sr((unsigned)o, it32, 5u);
            if (i > i_s) st4S(a.y3_n + o - g.p2, y3n4, sr);
            if (own) {
                st4S(a.s_n + o, sp4, sr);
                st4S(a.t_n + o, tp4, sr);
                st4S(a.q_n + o, qn4, sr);
            }
            y3m = y34;
            y3prev = y34;
            tprev = tb4;
        }
        // the last row has D_v t' = 0: y3 is unchanged there
        if (i_own == g.n1) {
            SRStream sr((unsigned)g.at(b, g.n1 - 1, j), it32, 6u);
            st4S(a.y3_n + g.at(b, g.n1 - 1, j), y3prev, sr);
        }
    }
    const double q2 = block_sum(aq.value(), red_d);
    const double du2 = block_sum(adu.value(), red_d);
    const double u2 = block_sum(au.value(), red_d);
    const int cta = a.sp.cta_base + bid;
    const int ncta = a.sp.cta_total > 0 ? a.sp.cta_total : nblk;
    if (threadIdx.x == 0) {
        a.part[3 * cta] = q2;
        a.part[3 * cta + 1] = du2;
        a.part[3 * cta + 2] = u2;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(&a.sc->k2_ticket, 1u) == (unsigned)(ncta - 1));
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double s0 = 0, s1 = 0, s2 = 0;
    for (int k = threadIdx.x; k < ncta; k += NT) {
        s0 += __ldcg(a.part + 3 * k);
        s1 += __ldcg(a.part + 3 * k + 1);
        s2 += __ldcg(a.part + 3 * k + 2);
    }
    s0 = block_sum(s0, red_d);
    s1 = block_sum(s1, red_d);
    s2 = block_sum(s2, red_d);
    if (threadIdx.x == 0) {
        Scal* sc = a.sc;
        double c = 1.0;
        if (!isfinite(s0) || !isfinite(s1) || !isfinite(s2)) {
            sc->error |= 1;
        } else if (s0 > 0.0) {
            c = fmin(1.0, P.eps * (double)P.gamma_y4 / sqrt(s0));
        }
        sc->c[P.parity ^ 1] = c;
        sc->q2 = s0;
        sc->du2 = s1;
        sc->u2 = s2;
        sc->iter++;
        sc->k2_ticket = 0;
        // the stopping rule of a batch cube (Eq. 28, or the pass cap): on the
        // device, so that a batch runs as one graph without host polling
        if (P.max_iter > 0) {
            const bool at_check = P.tol > 0.0 && P.check_every > 0 && sc->iter % P.check_every == 0;
            const bool conv = at_check && s2 > 0.0 && sqrt(s1 / s2) < P.tol;
            if (conv || sc->iter >= P.max_iter) {
                sc->done = 1;
                sc->stop_parity = P.parity ^ 1;
                if (P.live) atomicSub(P.live, 1);
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(NT, 3) k2_light(const K2Args<T> a) {
    k2_body(a, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// value sources of the radix search: the cube's s~, t~ or a flat vector
// ---------------------------------------------------------------------------
template <typename T>
struct CubeSrc {
    Geom g;
    const T *s, *t, *y3, *q;
    const Scal* sc;
    int parity;
    float gs, gt;
    int o0, nb;         // the stored bands [o0, o0 + nb) this launch visits
    // Calls f(valid, |s~|, |t~|) for every voxel this thread owns, four
    // columns at a time in row order; every lane of a warp makes the same
    // number of calls (warp-collective work inside f is allowed).  want_s /
    // want_t: whether the pass needs |s~| / |t~| (uniform over the launch); the
    // inputs of a vector not wanted are not read, and its value passed to f is
    // meaningless.
    template <typename F>
    __device__ void visit(const int bid, const int nblk, F&& f, const bool want_s, const bool want_t) const {
        const float cs = (float)(1.0 - sc->c[parity]);
        const unsigned quads = (unsigned)g.p2 / 4u;
        const unsigned n1 = (unsigned)g.n1;
        const unsigned total = (unsigned)nb * n1 * quads;       // < 2^31 for any cube that fits
        const unsigned row0 = (unsigned)o0 * n1;
        for (unsigned base = bid * blockDim.x; base < total; base += nblk * blockDim.x) {
            const unsigned item = base + threadIdx.x;
            const bool live = item < total;
            const unsigned row = row0 + (live ? item / quads : 0u);   // b * n1 + i
            const int j = (int)(item - (row - row0) * quads) * 4;
            const int i = (int)(row % n1);
            float4 s4 = make_float4(0, 0, 0, 0), t4 = s4, y34 = s4, yu4 = s4, q4 = s4;
            if (live) {
                const long long o = (long long)row * g.p2 + j;
                if (want_s) s4 = Vec4<T>::ld(s + o);
                if (want_t) {
                    t4 = Vec4<T>::ld(t + o);
                    y34 = Vec4<T>::ld(y3 + o);
                    if (i >= 1) yu4 = Vec4<T>::ld(y3 + o - g.p2);
                }
                q4 = Vec4<T>::ld(q + o);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float xs = 0.f, xt = 0.f;
                const bool valid = live && j + k < g.n2;
                if (valid)
                    s_t_tilde(comp(s4, k), comp(t4, k), comp(y34, k), comp(yu4, k), comp(q4, k), cs, i, g.n1,
                              gs, gt, xs, xt);
                f(valid, fabsf(xs), fabsf(xt));
            }
        }
    }
};

struct FlatSrc {
    const float* x;
    long long n;
    template <typename F>
    __device__ void visit(const int bid, const int nblk, F&& f, bool, bool) const {
        for (long long base = bid * (long long)blockDim.x; base < n; base += (long long)nblk * blockDim.x) {
            const long long l = base + threadIdx.x;
            const bool valid = l < n;
            f(valid, valid ? fabsf(x[l]) : 0.f, 0.f);
        }
    }
};

struct SearchArgs {
    Scal* sc;
    L1Work w;
    int nvec;        // 2 for the cube (s, t), 1 for a flat vector
    int cta_base = 0, cta_total = 0;   // this launch's CTAs among the stage's (0: alone)
    __device__ int total(int nblk) const { return cta_total > 0 ? cta_total : nblk; }
};

// Radix histogram pass of one level for every vector that needs it; the last
// CTA selects the bracket.
template <typename Src>
__device__ __forceinline__ void radix_body(const Src& src, const SearchArgs& a, const int level, const int bid,
                                           const int nblk) {
    extern __shared__ __align__(16) unsigned hsm[];   // [2][2048] counts, low and high residue halves
    __shared__ double sh_d[NT];
    __shared__ unsigned long long sh_u[NT];
    __shared__ int sh_i[1];
    __shared__ int is_last;
    const int want = NEED_RADIX0 + level;
    bool need[2];
    need[0] = a.sc->ctl[0].need == want;
    need[1] = a.nvec > 1 && a.sc->ctl[1].need == want;
    if (!need[0] && !need[1]) return;
    const RadixLevel lv{level};
    const int nb = lv.nbins();
    // 32-bit shared bins: count, and the residue split into its low and high
    // 10 bits so that a CTA's sums stay below 2^32 (it sees at most 2^21
    // values per vector, each half below 2^10); every add is fire-and-forget,
    // so no lane waits on a result
    unsigned* hc = hsm;
    unsigned* hrl = hsm + 2 * kHistBins;
    unsigned* hrh = hsm + 4 * kHistBins;
    for (int k = threadIdx.x; k < 6 * kHistBins; k += NT) hsm[k] = 0;
    __syncthreads();
    const unsigned pre0 = a.sc->ctl[0].prefix, pre1 = a.sc->ctl[1].prefix;
    auto insert = [&](int v, bool take, unsigned key) {
        if (take) {
            const int bn = v * kHistBins + lv.bin(key);
            const unsigned r = lv.residue(key);
            atomicAdd(hc + bn, 1u);
            if (r) {
                atomicAdd(hrl + bn, r & 1023u);
                atomicAdd(hrh + bn, r >> 10);
            }
        }
    };
    src.visit(bid, nblk, [&](bool valid, float x0, float x1) {
        if (need[0]) {
            const unsigned key = __float_as_uint(x0);
            insert(0, valid && lv.inside(key, pre0), key);
        }
        if (need[1]) {
            const unsigned key = __float_as_uint(x1);
            insert(1, valid && lv.inside(key, pre1), key);
        }
    }, need[0], need[1]);
    __syncthreads();
    for (int k = threadIdx.x; k < 2 * kHistBins; k += NT) {
        if ((k % kHistBins) >= nb) continue;
        if (hc[k]) atomicAdd(a.w.hcnt + k, (unsigned long long)hc[k]);
        const unsigned long long res = ((unsigned long long)hrh[k] << 10) + hrl[k];
        if (res) atomicAdd(a.w.hres + k, res);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(&a.sc->fb_ticket, 1u) == (unsigned)(a.total(nblk) - 1));
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    for (int v = 0; v < 2; ++v) {
        if (!need[v]) continue;
        l1_radix_select(a.sc->ctl[v], lv, a.w.hcnt + v * kHistBins, a.w.hres + v * kHistBins,
                        a.sc->radius[v], sh_d, sh_u, sh_i);
    }
    for (int k = threadIdx.x; k < 2 * kHistBins; k += NT) { a.w.hcnt[k] = 0; a.w.hres[k] = 0; }
    if (threadIdx.x == 0) a.sc->fb_ticket = 0;
}

template <typename Src>
__global__ void __launch_bounds__(NT) k_radix(const Src src, const SearchArgs a, const int level) {
    radix_body(src, a, level, blockIdx.x, gridDim.x);
}

// Candidates of one CTA collected in shared memory and appended to the global
// lists with one atomic per vector at the end of the pass (a warp-level global
// atomic per candidate serialises on the counter once windows are wide).
// What overflows the shared buffer goes straight to the global list.
constexpr int kBlkCand = 1024;
struct BlockCand {
    float (*buf)[kBlkCand];
    unsigned* cnt;     // [2]
    unsigned* base;    // [2]
    // the lists' key histograms over the windows (null: not kept)
    unsigned* nh[2] = {nullptr, nullptr};
    unsigned* nbinned = nullptr;
    NarrowGeom ng[2];
    __device__ void init() {
        if (threadIdx.x < 2) cnt[threadIdx.x] = 0;
        __syncthreads();
    }
    // keep vector v's list histogram over the key window (lo, hi]
    __device__ void keep_hist(const L1Work& w, int v, float lo, float hi) {
        ng[v] = narrow_geom(__float_as_uint(lo), __float_as_uint(hi));
        nh[v] = w.nh && ng[v].ok ? w.nh + v * 3 * kNarrowBins : nullptr;
        nbinned = w.nbinned;
    }
    // values past the buffer go straight to the global list and its histogram
    __device__ void append(int v, bool take, float x, float* gcand, unsigned* gcnt) {
        const unsigned mask = __ballot_sync(0xffffffffu, take);
        if (mask == 0) return;
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(mask) - 1;
        unsigned b = 0;
        if (lane == leader) b = atomicAdd(cnt + v, (unsigned)__popc(mask));
        b = __shfl_sync(0xffffffffu, b, leader);
        const unsigned k = b + __popc(mask & ((1u << lane) - 1u));
        if (take && k < (unsigned)kBlkCand) buf[v][k] = x;
        if (b + __popc(mask) > (unsigned)kBlkCand) {
            const bool over = take && k >= (unsigned)kBlkCand;
            append_candidate(over, x, gcand, gcnt);
            if (over && nh[v]) {
                narrow_add(nh[v], ng[v], __float_as_uint(x));
                atomicAdd(nbinned + v, 1u);
            }
        }
    }
    // whole block; before the pass's completion ticket
    __device__ void flush(float* const* gcand, Scal* sc) {
        __syncthreads();
        if (threadIdx.x < 2) {
            const unsigned n = min(cnt[threadIdx.x], (unsigned)kBlkCand);
            base[threadIdx.x] = n ? atomicAdd(&sc->acc[threadIdx.x].m, n) : 0u;
        }
        __syncthreads();
        for (int v = 0; v < 2; ++v) {
            const unsigned n = min(cnt[v], (unsigned)kBlkCand);
            for (unsigned k = threadIdx.x; k < n; k += blockDim.x)
                if (base[v] + k < kCandCap) gcand[v][base[v] + k] = buf[v][k];
        }
    }
    // after flush: counts the buffered candidates of vector v into the list's
    // key histogram (kept by keep_hist)
    __device__ void bin(int v) {
        if (!nh[v]) return;
        const unsigned n = min(cnt[v], (unsigned)kBlkCand);
        for (unsigned k = threadIdx.x; k < n; k += blockDim.x) narrow_add(nh[v], ng[v], __float_as_uint(buf[v][k]));
        if (threadIdx.x == 0 && n) atomicAdd(nbinned + v, n);
    }
};
#define GSSTV_BLOCK_CAND(name)                                   \
    __shared__ float name##_buf[2][kBlkCand];                    \
    __shared__ unsigned name##_cnt[2], name##_base[2];           \
    BlockCand name{name##_buf, name##_cnt, name##_base};         \
    name.init()

// Gathers the bracket bin of every vector that needs it (k_search_finish
// finishes tau).
template <typename Src>
__device__ __forceinline__ void gather_body(const Src& src, const SearchArgs& a, const int bid, const int nblk) {
    bool need[2];
    need[0] = a.sc->ctl[0].need == NEED_GATHER;
    need[1] = a.nvec > 1 && a.sc->ctl[1].need == NEED_GATHER;
    if (!need[0] && !need[1]) return;
    const float lo0 = a.sc->ctl[0].g_lo, hi0 = a.sc->ctl[0].g_hi;
    const float lo1 = a.sc->ctl[1].g_lo, hi1 = a.sc->ctl[1].g_hi;
    GSSTV_BLOCK_CAND(bc);
    if (need[0]) bc.keep_hist(a.w, 0, lo0, hi0);
    if (need[1]) bc.keep_hist(a.w, 1, lo1, hi1);
    src.visit(bid, nblk, [&](bool valid, float x0, float x1) {
        if (need[0]) bc.append(0, valid && x0 > lo0 && x0 <= hi0, x0, a.w.cand[0], &a.sc->acc[0].m);
        if (need[1]) bc.append(1, valid && x1 > lo1 && x1 <= hi1, x1, a.w.cand[1], &a.sc->acc[1].m);
    }, need[0], need[1]);
    bc.flush(a.w.cand, a.sc);
    bc.bin(0);
    bc.bin(1);
}

template <typename Src>
__global__ void __launch_bounds__(NT) k_gather(const Src src, const SearchArgs a) {
    gather_body(src, a, blockIdx.x, gridDim.x);
}

// One windowed pass after K1's window missed: count and sum of |x| above the
// retry window and its values as candidates (k_search_finish runs Michelot's
// finish; a second miss leaves the threshold to the radix passes).  Per-CTA
// partial sums go to pn / ps (the stencil pass's partial arrays, free by now).
template <typename Src>
__device__ __forceinline__ void window_body(const Src& src, const SearchArgs& a, unsigned long long* pn, double* ps,
                                            const int bid, const int nblk) {
    __shared__ double red_d[64];
    __shared__ unsigned long long red_u[64];
    bool need[2];
    need[0] = a.sc->ctl[0].need == NEED_WINDOW;
    need[1] = a.nvec > 1 && a.sc->ctl[1].need == NEED_WINDOW;
    if (!need[0] && !need[1]) return;
    const float lo0 = a.sc->ctl[0].g_lo, hi0 = a.sc->ctl[0].g_hi;
    const float lo1 = a.sc->ctl[1].g_lo, hi1 = a.sc->ctl[1].g_hi;
    WinAcc w0, w1;
    GSSTV_BLOCK_CAND(bc);
    if (need[0]) bc.keep_hist(a.w, 0, lo0, hi0);
    if (need[1]) bc.keep_hist(a.w, 1, lo1, hi1);
    src.visit(bid, nblk, [&](bool valid, float x0, float x1) {
        if (need[0]) {
            const bool hi = valid && x0 > hi0;
            if (hi) { w0.n++; w0.s.add(x0); }
            bc.append(0, valid && !hi && x0 > lo0, x0, a.w.cand[0], &a.sc->acc[0].m);
        }
        if (need[1]) {
            const bool hi = valid && x1 > hi1;
            if (hi) { w1.n++; w1.s.add(x1); }
            bc.append(1, valid && !hi && x1 > lo1, x1, a.w.cand[1], &a.sc->acc[1].m);
        }
    }, need[0], need[1]);
    bc.flush(a.w.cand, a.sc);
    bc.bin(0);
    bc.bin(1);
    float2* pbuf = reinterpret_cast<float2*>(red_d);
    const unsigned long long n0 = block_sum(w0.n, red_u), n1 = block_sum(w1.n, red_u);
    const double s0 = block_sum_pair(w0.s, pbuf), s1 = block_sum_pair(w1.s, pbuf);
    const int cta = a.cta_base + bid;
    if (threadIdx.x == 0) {
        pn[2 * cta] = n0; pn[2 * cta + 1] = n1;
        ps[2 * cta] = s0; ps[2 * cta + 1] = s1;
    }
}

template <typename Src>
__global__ void __launch_bounds__(NT) k_window(const Src src, const SearchArgs a, unsigned long long* pn,
                                               double* ps) {
    window_body(src, a, pn, ps, blockIdx.x, gridDim.x);
}

// The finish of K1's window (mode 2), of the retry window (mode 0) or of the
// gathered radix bracket (mode 1) of vector v, if it needs it: one CTA of kFinishThreads threads,
// the candidates staged in its shared memory when they fit (kFinishStage
// floats), narrowed on the float keys and finished by Michelot's step (see
// l1_window_finish).  A single CTA walking a list of a few hundred thousand
// candidates is bound by the latency of its loads, so it runs apart from the
// main pass with the most threads a CTA can have, and the vectors' searches
// (independent) run in CTAs of their own.  parts: the main pass's CTAs (mode
// 0: their count and sum above the window in pn / ps, two per CTA; mode 2:
// K1's four per CTA, the window's and the histogram's above-range statistics
// of both vectors).
constexpr int kFinishThreads = 1024;
constexpr unsigned kFinishStage = 32768;

// K1's window of vector v, after the fused pass: the CTAs' counts and sums
// above the window summed, tau found on the candidates (l1_window_finish); on
// a miss, K1's sampled histogram (when it was on) brackets tau for one retry
// pass, else the next window is placed from the bounds the miss gives or the
// radix passes run.  The whole block; K1's partials: pn / ps, four per CTA.
__device__ __noinline__ void k1_window_finish(const SearchArgs& a, const unsigned long long* pn, const double* ps,
                                              int parts, const int v, float* fstage, unsigned* scr, double* red_d,
                                              unsigned long long* red_u) {
    __shared__ int sh_flag;
    L1Ctl& C = a.sc->ctl[v];
    const double r = a.sc->radius[v];
    if (!(r > 0.0)) {
        if (threadIdx.x == 0) {
            C.tau = __int_as_float(0x7f800000);
            C.have_tau = 1;
            C.need = NEED_NONE;
            C.window_ok = 0;
        }
        return;
    }
    if (!__ldcg(&a.sc->k1_win[v])) {
        if (threadIdx.x == 0) {
            C.need = NEED_RADIX0; C.prefix = 0; C.n_above = 0; C.s_above = 0.0; C.exact_runs++;
        }
        return;
    }
    const bool hist_v = __ldcg(&a.sc->k1_hist[v]) != 0;
    unsigned long long n = 0, hn = 0;
    double s = 0.0, hs = 0.0;
    for (int k = threadIdx.x; k < parts; k += blockDim.x) {
        n += __ldcg(pn + 4 * k + v);
        s += __ldcg(ps + 4 * k + v);
        hn += __ldcg(pn + 4 * k + 2 + v);
        hs += __ldcg(ps + 4 * k + 2 + v);
    }
    n = block_sum(n, red_u);
    s = block_sum(s, red_d);
    const unsigned m = __ldcg(&a.sc->acc[v].m);
    const double tlo = C.theta_lo, thi = C.theta_hi;
    double tau = 0.0;
    WinInfo wi;
    const int miss = l1_window_finish((double)n, s, a.w.cand[v], m, tlo, thi, r, &tau, red_d, red_u, &wi, fstage,
                                      kFinishStage, scr, narrow_pre(a.w, v, m));
    narrow_clear(a.w, v);
    int hist_hit = 0;
    float h_lo = 0.f, h_hi = 0.f;
    double h_m = 0.0;
    if (miss && hist_v) {
        hn = block_sum(hn, red_u);
        hs = block_sum(hs, red_d);
        hist_hit = l1_hist_bracket(a.w.khist + v * kK1Bins, C.hbase, (double)hn, hs, r, (double)kHistSample,
                                   &h_lo, &h_hi, &h_m, &sh_flag, reinterpret_cast<unsigned*>(fstage));
    }
    if (hist_v) {
        __syncthreads();
        for (int k = threadIdx.x; k < kK1Bins; k += blockDim.x) a.w.khist[v * kK1Bins + k] = 0u;
    }
    if (threadIdx.x == 0) {
        if (!miss) {
            l1_record_tau(C, tau, (double)min(m, kCandCap), thi - tlo, true);
            C.hits++;
            if (C.hist_left > 0) C.hist_left--;
        } else if (hist_hit) {
            C.prefix = 0; C.n_above = 0; C.s_above = 0.0;
            C.need = NEED_WINDOW;
            C.g_lo = h_lo;
            C.g_hi = h_hi;
            C.hist_left = kHistPasses;
        } else {
            l1_after_miss(C, miss, wi, (double)n, m, tlo, thi);
        }
        a.sc->acc[v].m = 0;
    }
    __syncthreads();
}

constexpr size_t kFinishSmem = kFinishStage * sizeof(float) + 3 * kNarrowBins * sizeof(unsigned);
__device__ __forceinline__ void finish_body(const SearchArgs& a, int mode, const unsigned long long* pn,
                                            const double* ps, int parts, const int v) {
    extern __shared__ __align__(16) float fstage[];         // kFinishStage floats + the narrowing scratch
    __shared__ double red_d[64];
    __shared__ unsigned long long red_u[64];
    const int want = mode == 0 ? NEED_WINDOW : NEED_GATHER;
    unsigned* scr = reinterpret_cast<unsigned*>(fstage + kFinishStage);
    if (v >= a.nvec) return;
    if (mode == 2) {
        k1_window_finish(a, pn, ps, parts, v, fstage, scr, red_d, red_u);
        return;
    }
    {
        L1Ctl& C = a.sc->ctl[v];
        if (C.need != want) return;                         // uniform over the CTA
        const double r = a.sc->radius[v];
        const unsigned m = __ldcg(&a.sc->acc[v].m);
        const double lo = C.g_lo, hi = C.g_hi;
        double n = 0.0, sm = 0.0;
        if (mode == 0) {
            unsigned long long nn = 0;
            double ss = 0.0;
            for (int k = threadIdx.x; k < parts; k += blockDim.x) {
                nn += __ldcg(pn + 2 * k + v);
                ss += __ldcg(ps + 2 * k + v);
            }
            n = (double)block_sum(nn, red_u);
            sm = block_sum(ss, red_d);
        } else {
            n = (double)C.n_above;
            sm = C.s_above;
        }
        double tau = 0.0;
        const int rc = l1_window_finish(n, sm, a.w.cand[v], m, lo, hi, r, &tau, red_d, red_u, nullptr, fstage,
                                        kFinishStage, scr, narrow_pre(a.w, v, m));
        narrow_clear(a.w, v);
        if (threadIdx.x == 0) {
            if (mode == 0) {
                if (rc == 0) {
                    l1_record_tau(C, tau, (double)min(m, kCandCap), hi - lo, false);
                    C.retry_hits++;
                } else {
                    C.need = NEED_RADIX0; C.prefix = 0; C.n_above = 0; C.s_above = 0.0;
                    C.exact_runs++;
                }
            } else {
                if (rc == 2 && n > 0.0) {
                    // the root lies between the largest value of the bin and
                    // the next bin's edge: every value of the bin is inactive
                    tau = (sm - r) / n;
                } else if (rc != 0) {
                    atomicOr(&a.sc->error, 2);
                }
                l1_record_tau(C, tau, (double)min(m, kCandCap), hi - lo, false);
            }
            a.sc->acc[v].m = 0;
        }
        __syncthreads();
    }
}

// one CTA per vector
// After K1's window finish (mode 2) in a graph: the last of the launch's
// CTAs opens the conditional node of the search launches when a cube still
// needs a search (one thread, so that no two calls race).  need_any() reads the
// cubes' flags after every CTA's have landed.
template <typename F>
__device__ __forceinline__ void finish_gate(Scal* counter, unsigned total, cudaGraphConditionalHandle cond,
                                            F&& need_any) {
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&counter->fin_ticket, 1u) == total - 1u;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        counter->fin_ticket = 0u;
        const unsigned need = need_any() ? 1u : 0u;
        if (need) counter->gate_opens++;
        cudaGraphSetConditional(cond, need);
    }
}
__device__ __forceinline__ bool scal_needs_search(const Scal* s) {
    return !__ldcg(&s->done) && (__ldcg(&s->ctl[0].need) != NEED_NONE || __ldcg(&s->ctl[1].need) != NEED_NONE);
}

// one CTA per vector; gated: a graph's conditional node waits on this launch
__global__ void __launch_bounds__(kFinishThreads) k_search_finish(const SearchArgs a, int mode,
                                                                   const unsigned long long* pn,
                                                                   const double* ps, int parts, int gated,
                                                                   cudaGraphConditionalHandle cond) {
    finish_body(a, mode, pn, ps, parts, blockIdx.x);
    if (gated) finish_gate(a.sc, gridDim.x, cond, [&] { return scal_needs_search(a.sc); });
}

// out = soft(x, tau) for the standalone projection
__global__ void k_apply_flat(const float* x, float* out, long long n, const Scal* sc) {
    const double tau = sc->ctl[0].tau;
    const float tf = (float)tau;
    for (long long l = blockIdx.x * (long long)NT + threadIdx.x; l < n; l += (long long)gridDim.x * NT)
        out[l] = tau > 0.0 ? soft(x[l], tf) : x[l];
}

// ---------------------------------------------------------------------------
// layout conversion: (ncubes, n3, n1, *) arrays between pitches and types
// ---------------------------------------------------------------------------
// Cube by cube, 32 x 8 threads: a warp takes 32 columns of one row, blocks in
// y walk the rows (no division per element).
template <typename S, typename D>
__global__ void __launch_bounds__(256) k_convert(const S* src, long long src_pitch, long long src_cube, D* dst,
                                                 long long dst_pitch, long long dst_cube, int n1, int n2, int n3,
                                                 int ncubes, const double* scale) {
    const float f = scale ? (float)(1.0 - *scale) : 1.f;
    const long long rows = (long long)n3 * n1;
    for (int cb = 0; cb < ncubes; ++cb) {
        for (long long row = blockIdx.y * 8ll + threadIdx.y; row < rows; row += gridDim.y * 8ll) {
            const S* s = src + cb * src_cube + row * src_pitch;
            D* d = dst + cb * dst_cube + row * dst_pitch;
            for (int j = blockIdx.x * 32 + threadIdx.x; j < n2; j += gridDim.x * 32) {
                const float x = ldT(s + j);
                stT(d + j, scale ? f * x : x);
            }
        }
    }
}

// The same for float32 rows whose pitches, width and bases are multiples of
// four floats: one float4 per thread and row (more bytes in flight).
__global__ void __launch_bounds__(256) k_convert4(const float4* src, long long src_pitch, long long src_cube,
                                                  float4* dst, long long dst_pitch, long long dst_cube,
                                                  long long rows, int w4, int ncubes, const double* scale) {
    const float f = scale ? (float)(1.0 - *scale) : 1.f;
    for (int cb = 0; cb < ncubes; ++cb) {
        for (long long row = blockIdx.y * 8ll + threadIdx.y; row < rows; row += gridDim.y * 8ll) {
            const float4* s = src + cb * src_cube + row * src_pitch;
            float4* d = dst + cb * dst_cube + row * dst_pitch;
            for (int j = blockIdx.x * 32 + threadIdx.x; j < w4; j += gridDim.x * 32) {
                float4 x = __ldg(s + j);
                if (scale) { x.x *= f; x.y *= f; x.z *= f; x.w *= f; }
                d[j] = x;
            }
        }
    }
}

// All 21 float32 cubes of a state in one launch (grid z = cube), float4 rows;
// the last cube (q) is scaled by 1 - c into y4.
struct CubeCopy4 {
    const float4* src;
    float4* dst;
    int scaled;
};
struct StateCopy4 {
    CubeCopy4 c[21];
    long long rows, src_pitch, dst_pitch;   // pitches in float4
    int w4;
    const double* scale;
};

__global__ void __launch_bounds__(256) k_unpack_state4(const StateCopy4 a) {
    const CubeCopy4 cc = a.c[blockIdx.z];
    const float f = cc.scaled ? (float)(1.0 - *a.scale) : 1.f;
    for (long long row = blockIdx.y * 8ll + threadIdx.y; row < a.rows; row += gridDim.y * 8ll) {
        const float4* s = cc.src + row * a.src_pitch;
        float4* d = cc.dst + row * a.dst_pitch;
        for (int j = blockIdx.x * 32 + threadIdx.x; j < a.w4; j += gridDim.x * 32) {
            float4 x = __ldg(s + j);
            if (cc.scaled) { x.x *= f; x.y *= f; x.z *= f; x.w *= f; }
            d[j] = x;
        }
    }
}

int grid_for(long long n) {
    long long b = (n + NT - 1) / NT;
    return (int)std::max(1ll, std::min(b, device_sms() * 16ll));
}

// voxels a part's launch visits
long long part_voxels(const Geom& g, const SlabPart& sp) {
    return (long long)(sp.o1 - sp.o0) * g.n1 * g.n2;
}

int k2_grid_part(const Geom& g, const SlabPart& sp) {
    const long long items = (long long)(sp.o1 - sp.o0) * ((g.n1 + K2_ROWS - 1) / K2_ROWS) * (g.p2 / 4);
    return grid_for(items);
}

int radix_grid_n(long long n) {
    // enough CTAs that none sees more than 2^21 values (the shared bins are 32-bit)
    const long long min_ctas = (n + (1ll << 21) - 1) >> 21;
    return (int)std::max<long long>(std::min(grid_for(n), device_sms() * 3), min_ctas);
}

int gather_grid_n(long long n) { return std::min(grid_for(n), device_sms() * 4); }

template <typename T>
int launch_k2_t(const Geom& g, const IterBufs& b, const IterParams& p, Scal* sc, double* part,
                int part_cap, const SlabPart& sp, cudaStream_t st) {
    K2Args<T> a;
    a.g = g;
    a.u = (const T*)b.u; a.u_n = (const T*)b.u_n; a.s = (const T*)b.s; a.t = (const T*)b.t;
    a.y3 = (const T*)b.y3; a.q = (const T*)b.q; a.v = b.v;
    a.s_n = (T*)b.s_n; a.t_n = (T*)b.t_n; a.y3_n = (T*)b.y3_n; a.q_n = (T*)b.q_n;
    a.p = p;
    a.sc = sc;
    a.part = part;
    a.sp = sp;
    const int ctas = std::min(k2_grid_part(g, sp), part_cap);
    k2_light<T><<<ctas, NT, 0, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

template <typename Src>
int launch_radix_src(const Src& src, long long n, const SearchArgs& a, int level, cudaStream_t st) {
    const size_t smem = 6 * kHistBins * sizeof(unsigned);
    k_radix<Src><<<radix_grid_n(n), NT, smem, st>>>(src, a, level);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

template <typename T>
CubeSrc<T> make_cube_src(const Geom& g, const IterBufs& b, const IterParams& p, const Scal* sc,
                         const SlabPart& sp) {
    CubeSrc<T> c;
    c.g = g;
    c.s = (const T*)b.s; c.t = (const T*)b.t; c.y3 = (const T*)b.y3; c.q = (const T*)b.q;
    c.sc = sc;
    c.parity = p.parity;
    c.gs = p.gamma_s;
    c.gt = p.gamma_t;
    c.o0 = sp.o0;
    c.nb = sp.o1 - sp.o0;
    return c;
}

SearchArgs cube_args(Scal* sc, const L1Work& w, const SlabPart& sp) {
    SearchArgs a{sc, w, 2};
    a.cta_base = sp.cta_base;
    a.cta_total = sp.cta_total;
    return a;
}

template <typename T>
int launch_fallback_t(int level, const Geom& g, const IterBufs& b, const IterParams& p, Scal* sc,
                      const L1Work& w, const SlabPart& sp, cudaStream_t st) {
    const CubeSrc<T> src = make_cube_src<T>(g, b, p, sc, sp);
    return launch_radix_src(src, part_voxels(g, sp), cube_args(sc, w, sp), level, st);
}

template <typename T>
int launch_gather_t(const Geom& g, const IterBufs& b, const IterParams& p, Scal* sc, const L1Work& w,
                    const SlabPart& sp, cudaStream_t st) {
    const CubeSrc<T> src = make_cube_src<T>(g, b, p, sc, sp);
    k_gather<CubeSrc<T>><<<gather_grid_n(part_voxels(g, sp)), NT, 0, st>>>(src, cube_args(sc, w, sp));
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int window_grid_n(long long n, int part_cap) {
    return std::max(1, std::min({grid_for(n), device_sms() * 4, part_cap}));
}

template <typename T>
int launch_window_t(const Geom& g, const IterBufs& b, const IterParams& p, Scal* sc, const L1Work& w,
                    int part_cap, const SlabPart& sp, cudaStream_t st) {
    const CubeSrc<T> src = make_cube_src<T>(g, b, p, sc, sp);
    const int grid = window_grid_n(part_voxels(g, sp), part_cap);
    k_window<CubeSrc<T>><<<grid, NT, 0, st>>>(src, cube_args(sc, w, sp), w.k1_n, w.k1_s);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

template <typename S, typename D>
int launch_convert(const S* src, long long sp, long long sc_, D* dst, long long dp, long long dc,
                   const Geom& g, int ncubes, const double* scale, cudaStream_t st) {
    const long long rows = (long long)g.n3 * g.n1;
    if constexpr (std::is_same<S, float>::value && std::is_same<D, float>::value) {
        const bool a16 = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0;
        if (a16 && sp % 4 == 0 && dp % 4 == 0 && sc_ % 4 == 0 && dc % 4 == 0 && g.n2 % 4 == 0) {
            const int w4 = g.n2 / 4;
            const int gx = std::min((w4 + 31) / 32, 64);
            const long long gy = std::max(1ll, std::min({(rows + 7) / 8, (device_sms() * 16ll) / gx, 65535ll}));
            k_convert4<<<dim3(gx, (unsigned)gy), dim3(32, 8), 0, st>>>(
                reinterpret_cast<const float4*>(src), sp / 4, sc_ / 4, reinterpret_cast<float4*>(dst), dp / 4,
                dc / 4, rows, w4, ncubes, scale);
            return cudaGetLastError() == cudaSuccess ? 0 : -3;
        }
    }
    const int gx = std::min((g.n2 + 31) / 32, 64);
    const long long gy = std::max(1ll, std::min({(rows + 7) / 8, (device_sms() * 16ll) / gx, 65535ll}));
    k_convert<S, D><<<dim3(gx, (unsigned)gy), dim3(32, 8), 0, st>>>(src, sp, sc_, dst, dp, dc, g.n1, g.n2, g.n3,
                                                                    ncubes, scale);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ---------------------------------------------------------------------------
// batches: one launch of a stage for many cubes (float32 storage)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int batch_cube_of(const int* start, int n, int blk) {
    int lo = 0, hi = n - 1;                 // the last cube whose first CTA is <= blk
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= blk) lo = mid; else hi = mid - 1;
    }
    return lo;
}

struct SearchCube {
    CubeSrc<float> src;
    SearchArgs a;
    unsigned long long* pn;
    double* ps;
    int parts;
};
struct SearchBatchTab {
    int n;
    int start[kBatchMax + 1];
    SearchCube c[kBatchMax];
};
struct K2BatchTab {
    int n;
    int start[kBatchMax + 1];
    K2Args<float> c[kBatchMax];
};

__global__ void __launch_bounds__(NT) k_window_batch(const __grid_constant__ SearchBatchTab t) {
    const int c = batch_cube_of(t.start, t.n, blockIdx.x);
    const SearchCube& q = t.c[c];
    if (__ldcg(&q.a.sc->done)) return;
    window_body(q.src, q.a, q.pn, q.ps, blockIdx.x - t.start[c], t.start[c + 1] - t.start[c]);
}
__global__ void __launch_bounds__(NT) k_radix_batch(const __grid_constant__ SearchBatchTab t, const int level) {
    const int c = batch_cube_of(t.start, t.n, blockIdx.x);
    const SearchCube& q = t.c[c];
    if (__ldcg(&q.a.sc->done)) return;
    radix_body(q.src, q.a, level, blockIdx.x - t.start[c], t.start[c + 1] - t.start[c]);
}
__global__ void __launch_bounds__(NT) k_gather_batch(const __grid_constant__ SearchBatchTab t) {
    const int c = batch_cube_of(t.start, t.n, blockIdx.x);
    const SearchCube& q = t.c[c];
    if (__ldcg(&q.a.sc->done)) return;
    gather_body(q.src, q.a, blockIdx.x - t.start[c], t.start[c + 1] - t.start[c]);
}
// one CTA per cube and vector
__global__ void __launch_bounds__(kFinishThreads) k_finish_batch(const __grid_constant__ SearchBatchTab t,
                                                                  const int mode, int gated,
                                                                  cudaGraphConditionalHandle cond) {
    const SearchCube& q = t.c[blockIdx.x >> 1];
    if (!__ldcg(&q.a.sc->done)) finish_body(q.a, mode, q.pn, q.ps, q.parts, blockIdx.x & 1);
    // every CTA counts, a stopped cube's too (the first cube's scalars hold the count)
    if (gated)
        finish_gate(t.c[0].a.sc, gridDim.x, cond, [&] {
            bool any = false;
            for (int c = 0; c < t.n; ++c) any = any || scal_needs_search(t.c[c].a.sc);
            return any;
        });
}
__global__ void __launch_bounds__(NT, 3) k2_batch(const __grid_constant__ K2BatchTab t) {
    const int c = batch_cube_of(t.start, t.n, blockIdx.x);
    // by value: the table is indexed by a run-time cube, so each field is
    // loaded once instead of at each use
    const K2Args<float> a = t.c[c];
    if (__ldcg(&a.sc->done)) return;
    k2_body(a, blockIdx.x - t.start[c], t.start[c + 1] - t.start[c]);
}

// the search table of a stage; grid(q): CTAs of cube q's share
template <typename G>
int search_table(const BatchCube* cubes, int n, SearchBatchTab& t, G&& grid) {
    if (n < 1 || n > kBatchMax) return -1;
    static_assert(sizeof(SearchBatchTab) <= 32000, "kernel parameter space");
    t.n = n;
    int total = 0;
    for (int c = 0; c < n; ++c) {
        const BatchCube& q = cubes[c];
        const SlabPart whole = whole_cube(q.g);
        t.c[c].src = make_cube_src<float>(q.g, q.b, q.p, q.sc, whole);
        t.c[c].a = cube_args(q.sc, q.l1, whole);
        t.c[c].pn = q.l1.k1_n;
        t.c[c].ps = q.l1.k1_s;
        t.c[c].parts = window_grid_n(part_voxels(q.g, whole), q.k1_ctas);
        t.start[c] = total;
        total += grid(q, whole);
    }
    t.start[n] = total;
    return total;
}

}  // namespace

int device_sms() {
    constexpr int kMaxDev = 64;
    constexpr int kFallback = 152;     // GB300, if the query fails
    static std::once_flag once[kMaxDev];
    static int sms[kMaxDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
        cudaGetLastError();
        return kFallback;
    }
    std::call_once(once[dev], [dev] {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
            cudaGetLastError();
            n = kFallback;
        }
        sms[dev] = n;
    });
    return sms[dev];
}

int light_configure(int storage) {
    const int smem = 6 * kHistBins * sizeof(unsigned);
    cudaError_t e = cudaErrorInvalidValue;
    switch (storage) {
        case 0: e = cudaFuncSetAttribute(k_radix<CubeSrc<float>>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); break;
        case 1: e = cudaFuncSetAttribute(k_radix<CubeSrc<__nv_bfloat16>>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); break;
        case 2: e = cudaFuncSetAttribute(k_radix<CubeSrc<__half>>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); break;
    }
    if (e != cudaSuccess) return -3;
    e = cudaFuncSetAttribute(k_radix<FlatSrc>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return -3;
    e = cudaFuncSetAttribute(k_search_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, kFinishSmem);
    return e == cudaSuccess ? 0 : -3;
}

int launch_search_finish(int mode, Scal* sc, const L1Work& w, int nvec, const unsigned long long* pn,
                         const double* ps, int parts, cudaStream_t st, int gated,
                         cudaGraphConditionalHandle cond) {
    SearchArgs a{sc, w, nvec};
    k_search_finish<<<nvec, kFinishThreads, kFinishSmem, st>>>(a, mode, pn, ps, parts, gated, cond);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int k2_grid_ctas(const Geom& g) { return k2_grid_part(g, whole_cube(g)); }

int window_grid(const Geom& g, const SlabPart& sp, int part_cap) {
    return window_grid_n(part_voxels(g, sp), part_cap);
}
int radix_grid(const Geom& g, const SlabPart& sp) { return radix_grid_n(part_voxels(g, sp)); }
int gather_grid(const Geom& g, const SlabPart& sp) { return gather_grid_n(part_voxels(g, sp)); }
int k2_grid(const Geom& g, const SlabPart& sp, int part_cap) { return std::min(k2_grid_part(g, sp), part_cap); }

int launch_k2(int storage, const Geom& g, const IterBufs& b, const IterParams& p, Scal* sc,
              double* part, int part_cap, const SlabPart& sp, cudaStream_t st) {
    switch (storage) {
        case 0: return launch_k2_t<float>(g, b, p, sc, part, part_cap, sp, st);
        case 1: return launch_k2_t<__nv_bfloat16>(g, b, p, sc, part, part_cap, sp, st);
        case 2: return launch_k2_t<__half>(g, b, p, sc, part, part_cap, sp, st);
    }
    return -1;
}


int launch_fallback(int storage, int level, const Geom& g, const IterBufs& b, const IterParams& p,
                    Scal* sc, const L1Work& w, const SlabPart& sp, cudaStream_t st) {
    switch (storage) {
        case 0: return launch_fallback_t<float>(level, g, b, p, sc, w, sp, st);
        case 1: return launch_fallback_t<__nv_bfloat16>(level, g, b, p, sc, w, sp, st);
        case 2: return launch_fallback_t<__half>(level, g, b, p, sc, w, sp, st);
    }
    return -1;
}

int launch_gather(int storage, const Geom& g, const IterBufs& b, const IterParams& p, Scal* sc,
                  const L1Work& w, const SlabPart& sp, cudaStream_t st) {
    switch (storage) {
        case 0: return launch_gather_t<float>(g, b, p, sc, w, sp, st);
        case 1: return launch_gather_t<__nv_bfloat16>(g, b, p, sc, w, sp, st);
        case 2: return launch_gather_t<__half>(g, b, p, sc, w, sp, st);
    }
    return -1;
}

int launch_window(int storage, const Geom& g, const IterBufs& b, const IterParams& p, Scal* sc,
                  const L1Work& w, int part_cap, const SlabPart& sp, cudaStream_t st) {
    switch (storage) {
        case 0: return launch_window_t<float>(g, b, p, sc, w, part_cap, sp, st);
        case 1: return launch_window_t<__nv_bfloat16>(g, b, p, sc, w, part_cap, sp, st);
        case 2: return launch_window_t<__half>(g, b, p, sc, w, part_cap, sp, st);
    }
    return -1;
}

int launch_window_batch(const BatchCube* cubes, int n, cudaStream_t st) {
    SearchBatchTab t{};
    const int total = search_table(cubes, n, t, [](const BatchCube& q, const SlabPart& w) {
        return window_grid_n(part_voxels(q.g, w), q.k1_ctas);
    });
    if (total < 0) return -1;
    k_window_batch<<<total, NT, 0, st>>>(t);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_radix_batch(const BatchCube* cubes, int n, int level, cudaStream_t st) {
    SearchBatchTab t{};
    const int total = search_table(cubes, n, t, [](const BatchCube& q, const SlabPart& w) {
        return radix_grid_n(part_voxels(q.g, w));
    });
    if (total < 0) return -1;
    k_radix_batch<<<total, NT, 6 * kHistBins * sizeof(unsigned), st>>>(t, level);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_gather_batch(const BatchCube* cubes, int n, cudaStream_t st) {
    SearchBatchTab t{};
    const int total = search_table(cubes, n, t, [](const BatchCube& q, const SlabPart& w) {
        return gather_grid_n(part_voxels(q.g, w));
    });
    if (total < 0) return -1;
    k_gather_batch<<<total, NT, 0, st>>>(t);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// Whether any cube still needs a threshold search after K1's finish: sets the
// condition of the graph node that holds the search launches (one thread, so
// that no two calls race).
struct GateArgs {
    Scal* sc[kBatchMax];
    int n;
    cudaGraphConditionalHandle cond;
};
__global__ void k_search_gate(const __grid_constant__ GateArgs g) {
    if (threadIdx.x != 0) return;
    unsigned need = 0u;
    for (int c = 0; c < g.n; ++c) {
        const Scal* s = g.sc[c];
        if (__ldcg(&s->done)) continue;
        if (__ldcg(&s->ctl[0].need) != NEED_NONE || __ldcg(&s->ctl[1].need) != NEED_NONE) need = 1u;
    }
    if (need) g.sc[0]->gate_opens++;
    cudaGraphSetConditional(g.cond, need);
}

int launch_search_gate(Scal* const* sc, int n, cudaGraphConditionalHandle cond, cudaStream_t st) {
    if (n < 1 || n > kBatchMax) return -1;
    GateArgs g{};
    for (int c = 0; c < n; ++c) g.sc[c] = sc[c];
    g.n = n;
    g.cond = cond;
    k_search_gate<<<1, 32, 0, st>>>(g);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_finish_batch(const BatchCube* cubes, int n, int mode, cudaStream_t st, int gated,
                        cudaGraphConditionalHandle cond) {
    SearchBatchTab t{};
    if (search_table(cubes, n, t, [](const BatchCube&, const SlabPart&) { return 1; }) < 0) return -1;
    if (mode == 2)                       // K1's partials: one set per CTA of the cube's K1 grid
        for (int c = 0; c < n; ++c) t.c[c].parts = k1_tma_grid(cubes[c].g, whole_cube(cubes[c].g), cubes[c].k1_chunk);
    k_finish_batch<<<2 * n, kFinishThreads, kFinishSmem, st>>>(t, mode, gated, cond);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_k2_batch(const BatchCube* cubes, int n, cudaStream_t st) {
    if (n < 1 || n > kBatchMax) return -1;
    static_assert(sizeof(K2BatchTab) <= 32000, "kernel parameter space");
    K2BatchTab t{};
    t.n = n;
    int total = 0;
    for (int c = 0; c < n; ++c) {
        const BatchCube& q = cubes[c];
        K2Args<float>& a = t.c[c];
        a.g = q.g;
        a.u = (const float*)q.b.u; a.u_n = (const float*)q.b.u_n; a.s = (const float*)q.b.s;
        a.t = (const float*)q.b.t; a.y3 = (const float*)q.b.y3; a.q = (const float*)q.b.q; a.v = q.b.v;
        a.s_n = (float*)q.b.s_n; a.t_n = (float*)q.b.t_n; a.y3_n = (float*)q.b.y3_n; a.q_n = (float*)q.b.q_n;
        a.p = q.p;
        a.sc = q.sc;
        a.part = q.k2_part;
        a.sp = whole_cube(q.g);
        t.start[c] = total;
        total += std::min(k2_grid_part(q.g, a.sp), q.k2_cap);
    }
    t.start[n] = total;
    k2_batch<<<total, NT, 0, st>>>(t);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int k1_batch_configure();

int batch_configure() {
    if (k1_batch_configure() != 0) return -3;
    cudaError_t e = cudaFuncSetAttribute(k_radix_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(6 * kHistBins * sizeof(unsigned)));
    if (e != cudaSuccess) return -3;
    e = cudaFuncSetAttribute(k_finish_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFinishSmem);
    return e == cudaSuccess ? 0 : -3;
}

int launch_copy_f32(const float* src, long long src_pitch, long long src_cube, float* dst, long long dst_pitch,
                    long long dst_cube, int n1, int n2, int nbands, int ncubes, const double* scale,
                    cudaStream_t st) {
    if (nbands <= 0 || ncubes <= 0) return 0;
    Geom g{};
    g.n1 = n1; g.n2 = n2; g.n3 = nbands;
    return launch_convert(src, src_pitch, src_cube, dst, dst_pitch, dst_cube, g, ncubes, scale, st);
}

// dense float32 (ncubes, n3, n1, n2)  ->  pitched storage cubes
int launch_pack(int storage, const float* src, void* dst, const Geom& g, int ncubes, cudaStream_t st) {
    const long long sp = g.n2, scb = (long long)g.n3 * g.n1 * g.n2;
    switch (storage) {
        case 0: return launch_convert(src, sp, scb, (float*)dst, g.p2, g.cube, g, ncubes, nullptr, st);
        case 1: return launch_convert(src, sp, scb, (__nv_bfloat16*)dst, g.p2, g.cube, g, ncubes, nullptr, st);
        case 2: return launch_convert(src, sp, scb, (__half*)dst, g.p2, g.cube, g, ncubes, nullptr, st);
    }
    return -1;
}

// pitched float32 (the handle's v)  ->  pitched storage cube
int launch_pitched_to_storage(int storage, const float* src, void* dst, const Geom& g, cudaStream_t st) {
    switch (storage) {
        case 0: return launch_convert(src, g.p2, g.cube, (float*)dst, g.p2, g.cube, g, 1, nullptr, st);
        case 1: return launch_convert(src, g.p2, g.cube, (__nv_bfloat16*)dst, g.p2, g.cube, g, 1, nullptr, st);
        case 2: return launch_convert(src, g.p2, g.cube, (__half*)dst, g.p2, g.cube, g, 1, nullptr, st);
    }
    return -1;
}

// dense float32 (n3, n1, n2)  ->  pitched float32
int launch_dense_to_pitched(const float* src, float* dst, const Geom& g, cudaStream_t st) {
    return launch_convert(src, (long long)g.n2, (long long)g.n3 * g.n1 * g.n2, dst, g.p2, g.cube, g, 1,
                          nullptr, st);
}

int launch_unpack(int storage, const void* src, float* dst, const Geom& g, int ncubes, cudaStream_t st) {
    const long long dp = g.n2, dcb = (long long)g.n3 * g.n1 * g.n2;
    switch (storage) {
        case 0: return launch_convert((const float*)src, g.p2, g.cube, dst, dp, dcb, g, ncubes, nullptr, st);
        case 1: return launch_convert((const __nv_bfloat16*)src, g.p2, g.cube, dst, dp, dcb, g, ncubes, nullptr, st);
        case 2: return launch_convert((const __half*)src, g.p2, g.cube, dst, dp, dcb, g, ncubes, nullptr, st);
    }
    return -1;
}

int launch_unpack_state(int storage, const void* const src[9], float* const dst[9], const double* c,
                        const Geom& g, cudaStream_t st) {
    static const int ncubes[9] = {1, 1, 1, 6, 6, 2, 2, 1, 1};
    if (storage != 0 || g.n2 % 4 != 0) return 1;
    StateCopy4 a;
    const long long dense = (long long)g.n3 * g.n1 * g.n2;
    int k = 0;
    for (int f = 0; f < 9; ++f) {
        if (((reinterpret_cast<uintptr_t>(src[f]) | reinterpret_cast<uintptr_t>(dst[f])) & 15) != 0) return 1;
        for (int cb = 0; cb < ncubes[f]; ++cb, ++k) {
            a.c[k].src = reinterpret_cast<const float4*>(static_cast<const float*>(src[f]) + cb * g.cube);
            a.c[k].dst = reinterpret_cast<float4*>(dst[f] + cb * dense);
            a.c[k].scaled = f == 8;
        }
    }
    a.rows = (long long)g.n3 * g.n1;
    a.src_pitch = g.p2 / 4;
    a.dst_pitch = g.n2 / 4;
    a.w4 = g.n2 / 4;
    a.scale = c;
    const int gx = std::min((a.w4 + 31) / 32, 64);
    const long long gy = std::max(1ll, std::min({(a.rows + 7) / 8, (device_sms() * 16ll) / (gx * 21ll), 65535ll}));
    k_unpack_state4<<<dim3(gx, (unsigned)gy, 21), dim3(32, 8), 0, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_scale_unpack(int storage, const void* q, const double* c, float* dst, const Geom& g,
                        cudaStream_t st) {
    const long long dp = g.n2, dcb = (long long)g.n3 * g.n1 * g.n2;
    switch (storage) {
        case 0: return launch_convert((const float*)q, g.p2, g.cube, dst, dp, dcb, g, 1, c, st);
        case 1: return launch_convert((const __nv_bfloat16*)q, g.p2, g.cube, dst, dp, dcb, g, 1, c, st);
        case 2: return launch_convert((const __half*)q, g.p2, g.cube, dst, dp, dcb, g, 1, c, st);
    }
    return -1;
}

// ---------------------------------------------------------------------------
// standalone projection of a flat device vector onto an l1 ball
// ---------------------------------------------------------------------------
int l1_project_standalone(const float* x, long long n, double radius, float* out, double* tau,
                          cudaStream_t st) {
    if (light_configure(0) != 0) return -3;
    Scal* sc = nullptr;
    L1Work w{};
    size_t bytes_hist = 2 * kHistBins * sizeof(unsigned long long);
    int rc = 0;
    if (cudaMalloc(&sc, sizeof(Scal)) != cudaSuccess) return -2;
    if (cudaMalloc(&w.hcnt, bytes_hist) != cudaSuccess || cudaMalloc(&w.hres, bytes_hist) != cudaSuccess ||
        cudaMalloc(&w.cand[0], kCandCap * sizeof(float)) != cudaSuccess) {
        rc = -2;
    }
    if (rc == 0) {
        w.cand[1] = w.cand[0];
        Scal h{};
        h.radius[0] = radius;
        h.ctl[0].need = radius > 0.0 ? NEED_RADIX0 : NEED_NONE;
        h.ctl[0].tau = radius > 0.0 ? 0.0 : (double)INFINITY;
        if (cudaMemcpyAsync(sc, &h, sizeof(Scal), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemsetAsync(w.hcnt, 0, bytes_hist, st) != cudaSuccess ||
            cudaMemsetAsync(w.hres, 0, bytes_hist, st) != cudaSuccess)
            rc = -3;
        const FlatSrc src{x, n};
        const SearchArgs a{sc, w, 1};
        for (int level = 0; level < 3 && rc == 0; ++level) rc = launch_radix_src(src, n, a, level, st);
        if (rc == 0) {
            k_gather<FlatSrc><<<gather_grid_n(n), NT, 0, st>>>(src, a);
            k_search_finish<<<1, kFinishThreads, kFinishSmem, st>>>(a, 1, nullptr, nullptr, 0, 0, 0);
            k_apply_flat<<<grid_for(n), NT, 0, st>>>(x, out, n, sc);
            if (cudaGetLastError() != cudaSuccess) rc = -3;
        }
        if (rc == 0) {
            if (cudaMemcpyAsync(&h, sc, sizeof(Scal), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                rc = -3;
            else if (h.error) rc = -6;
            else if (tau) *tau = h.ctl[0].tau;
        }
    }
    cudaStreamSynchronize(st);
    cudaFree(sc);
    cudaFree(w.hcnt);
    cudaFree(w.hres);
    cudaFree(w.cand[0]);
    return rc;
}

}  // namespace gsstv

// ---------------------------------------------------------------------------
// Allocation-free l1-ball projection.
//
// Same kernels as gsstv_project_l1ball, but every scratch byte (controller
// block, radix histograms, candidate buffer) lives in one file-scope device
// array instead of cudaMalloc'd memory, for callers that are not allowed to
// allocate device memory.  The candidate buffer here holds
// GSSTV_NOALLOC_MAX_N values; a radix bracket never holds more values than
// the whole input, so every n <= GSSTV_NOALLOC_MAX_N fits, and larger n are
// refused.
// ---------------------------------------------------------------------------
#include <mutex>

#include "gsstv.h"

namespace gsstv {
namespace {

constexpr size_t kNaScal = (sizeof(Scal) + 255) / 256 * 256;
constexpr size_t kNaHist = 2 * kHistBins * sizeof(unsigned long long);
constexpr size_t kNaCand = (size_t)GSSTV_NOALLOC_MAX_N * sizeof(float);
constexpr size_t kNaBytes = kNaScal + 2 * kNaHist + kNaCand;

// The scratch array: on every device that loads this library, until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

constexpr int kMaxDevices = 64;
unsigned char* g_na_ptr[kMaxDevices] = {};     // device address of the array, per device
std::mutex g_na_mutex;

__global__ void k_noalloc_init(Scal* sc, double radius) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        Scal z;
        memset(&z, 0, sizeof(z));
        z.radius[0] = radius;
        z.ctl[0].need = radius > 0.0 ? NEED_RADIX0 : NEED_NONE;
        z.ctl[0].tau = radius > 0.0 ? 0.0 : (double)__int_as_float(0x7f800000);
        *sc = z;
    }
}

// Resolves the array's device address on the current device (first call on
// that device only) and configures the kernels it launches.
int noalloc_setup(unsigned char** base) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return -3;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return -3;
        if (light_configure(0) != 0) return -3;
        g_na_ptr[dev] = (unsigned char*)p;
    }
    *base = g_na_ptr[dev];
    return 0;
}

}  // namespace

int l1_project_noalloc(const float* x, long long n, double radius, float* out, double* tau,
                       cudaStream_t st) {
    unsigned char* base = nullptr;
    if (noalloc_setup(&base) != 0) return -3;
    Scal* sc = reinterpret_cast<Scal*>(base);
    L1Work w{};
    w.hcnt = reinterpret_cast<unsigned long long*>(base + kNaScal);
    w.hres = reinterpret_cast<unsigned long long*>(base + kNaScal + kNaHist);
    w.cand[0] = w.cand[1] = reinterpret_cast<float*>(base + kNaScal + 2 * kNaHist);
    // the previous call's contents stay in the array: clear what must start at zero
    k_noalloc_init<<<1, 32, 0, st>>>(sc, radius);
    if (cudaGetLastError() != cudaSuccess) return -3;
    if (cudaMemsetAsync(w.hcnt, 0, 2 * kNaHist, st) != cudaSuccess) return -3;
    const FlatSrc src{x, n};
    const SearchArgs a{sc, w, 1};
    for (int level = 0; level < 3; ++level)
        if (launch_radix_src(src, n, a, level, st) != 0) return -3;
    k_gather<FlatSrc><<<gather_grid_n(n), NT, 0, st>>>(src, a);
    k_search_finish<<<1, kFinishThreads, kFinishSmem, st>>>(a, 1, nullptr, nullptr, 0, 0, 0);
    k_apply_flat<<<grid_for(n), NT, 0, st>>>(x, out, n, sc);
    if (cudaGetLastError() != cudaSuccess) return -3;
    double t = 0.0;
    int err = 0;
    if (cudaMemcpyAsync(&t, &sc->ctl[0].tau, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&err, &sc->error, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return -3;
    if (err) return -6;
    if (tau) *tau = t;
    return 0;
}

}  // namespace gsstv

extern "C" int gsstv_project_l1ball_noalloc(const float* d_x, int64_t n, double radius, float* d_out,
                                            double* tau_out, void* stream) {
    if (!d_x || !d_out || n < 0 || !(radius >= 0.0) || !std::isfinite(radius)) return GSSTV_ERR_ARG;
    if (n > GSSTV_NOALLOC_MAX_N) return GSSTV_ERR_ARG;
    if (n == 0) { if (tau_out) *tau_out = 0.0; return GSSTV_OK; }
    const int rc = gsstv::l1_project_noalloc(d_x, (long long)n, radius, d_out, tau_out, (cudaStream_t)stream);
    return rc == 0 ? GSSTV_OK : rc == -6 ? GSSTV_ERR_INTERNAL : GSSTV_ERR_CUDA;
}
