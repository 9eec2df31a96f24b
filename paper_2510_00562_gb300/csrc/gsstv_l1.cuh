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

// Michelot's fixed point restricted to a window.  One whole block calls it.
// n_hi, s_hi: count and sum of |x| > theta_hi; cand[0..m_raw): every |x| in
// (theta_lo, theta_hi].  Returns 0 with *tau_out; 2 when the root lies above
// the window; 1 when it lies below or the candidates overflowed the buffer.
// stage (optional): shared memory for stage_cap floats that the block no
// longer uses; when the candidates fit they are copied there on the first
// pass and every later pass reads them from it instead of from L2.
static __device__ int l1_window_finish(double n_hi, double s_hi, const float* cand, unsigned m_raw,
                                       double theta_lo, double theta_hi, double r,
                                       double* tau_out, double* red_d,
                                       unsigned long long* red_u, WinInfo* info = nullptr,
                                       float* stage = nullptr, unsigned stage_cap = 0) {
    const double phi_hi = s_hi - n_hi * theta_hi - r;
    if (info) info->phi_hi = phi_hi;
    if (m_raw > kCandCap) return 1;
    const unsigned m = m_raw;
    if (phi_hi > 0.0) return 2;                        // root above the window
    const bool staged = stage && m <= stage_cap;
    Kahan ks;
    for (unsigned k = threadIdx.x; k < m; k += blockDim.x) {
        const float x = __ldcg(cand + k);
        if (staged) stage[k] = x;
        ks.add(x);
    }
    const double sum_c = block_sum(ks.value(), red_d);      // (its barriers publish the stage)
    const double n_all = n_hi + (double)m;
    const double phi_lo = s_hi + sum_c - n_all * theta_lo - r;
    if (info) { info->phi_lo = phi_lo; info->n_lo = n_all; }
    if (phi_lo < 0.0) {
        if (theta_lo <= 0.0) { *tau_out = 0.0; return 0; }  // inside the ball
        return 1;                                      // root below the window
    }
    double tau = (s_hi + sum_c - r) / n_all;
    unsigned long long prev = m;
    for (int it = 0; it < 200; ++it) {
        // for a float x, x > tau exactly when x > (tau rounded down to float):
        // the test runs in FP32 (GB300's FP64 rate is a small fraction of it)
        const float tf = __double2float_rd(tau);
        Kahan ka;
        unsigned long long c = 0;
        for (unsigned k = threadIdx.x; k < m; k += blockDim.x) {
            const float x = staged ? stage[k] : __ldcg(cand + k);
            if (x > tf) { ka.add(x); ++c; }
        }
        const double sa = block_sum(ka.value(), red_d);
        const unsigned long long ca = block_sum(c, red_u);
        const double tn = (s_hi + sa - r) / (n_hi + (double)ca);
        tau = tn;
        if (ca == prev) break;
        prev = ca;
    }
    *tau_out = tau;
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

// After K1's window missed: the bracket of the root that K1's histogram of
// |x| gives.  hist: kK1Bins counts, bin b holding the |x| in [e_b, e_{b+1})
// with e_b = hist_edge(hbase, b); n_top, s_top: count and sum of |x| >= e_top.
// Taking every binned value at its bin's lower (upper) edge bounds phi at each
// edge from below (above); the highest edge with phi >= 0 from below and the
// lowest edge above it with phi < 0 from above bracket the root.  Returns 1
// with the window (*lo, *hi] and the number of values inside it in *m, or 0
// when the range does not bracket the root (or more than kCandCap values sit
// in the bracket).  The bounds carry a relative margin, and the retry pass on
// the window computes everything exactly, so a wrong bracket costs only time.
// One whole block calls it; warp 0 works.
static __device__ int l1_hist_bracket(const unsigned* hist, unsigned hbase, double n_top, double s_top,
                                      double r, float* lo_out, float* hi_out, double* m_out, int* sh_i) {
    constexpr int PER = kK1Bins / 32;
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const int b0 = lane * PER;
        double c_l = 0.0, sl_l = 0.0, sh_l = 0.0;
        for (int b = b0; b < b0 + PER; ++b) {
            const double c = (double)__ldcg(hist + b);
            c_l += c;
            sl_l += c * (double)hist_edge(hbase, b);
            sh_l += c * (double)hist_edge(hbase, b + 1);
        }
        // totals of the lanes above this one (exclusive suffix)
        double c_in = c_l, sl_in = sl_l, sh_in = sh_l;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double c = __shfl_down_sync(0xffffffffu, c_in, o);
            const double a = __shfl_down_sync(0xffffffffu, sl_in, o);
            const double b = __shfl_down_sync(0xffffffffu, sh_in, o);
            if (lane + o < 32) { c_in += c; sl_in += a; sh_in += b; }
        }
        const double total_sh = __shfl_sync(0xffffffffu, sh_in, 0);
        // the float32-compensated sums carry about 1e-7 relative error
        const double margin = 1e-6 * (s_top + total_sh + r);
        const double top = (double)hist_edge(hbase, kK1Bins);
        const double phi_top = s_top - n_top * top - r;         // exact up to the sums' rounding
        // pass 1: the highest edge with phi >= margin from below
        double N = n_top + (c_in - c_l), SL = s_top + (sl_in - sl_l);
        int a_best = phi_top >= margin ? kK1Bins : -1;
        for (int b = b0 + PER - 1; b >= b0 && a_best < 0; --b) {
            const double e = (double)hist_edge(hbase, b);
            const double c = (double)__ldcg(hist + b);
            N += c;
            SL += c * e;
            if (SL - N * e - r >= margin) a_best = b;
        }
        int a_all = a_best;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a_all = max(a_all, __shfl_xor_sync(0xffffffffu, a_all, o));
        // pass 2: the lowest edge above it with phi < -margin from above
        int c_best = kK1Bins + 1;
        if (a_all >= 0 && a_all < kK1Bins) {
            if (phi_top < -margin) c_best = kK1Bins;
            N = n_top + (c_in - c_l);
            double SH = s_top + (sh_in - sh_l);
            for (int b = b0 + PER - 1; b >= b0; --b) {
                const double e = (double)hist_edge(hbase, b);
                const double c = (double)__ldcg(hist + b);
                N += c;
                SH += c * (double)hist_edge(hbase, b + 1);
                if (b > a_all && SH - N * e - r < -margin) c_best = b;   // the lowest such b of this lane
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c_best = min(c_best, __shfl_xor_sync(0xffffffffu, c_best, o));
        // values inside the bracket [e_a, e_c)
        double m = 0.0;
        if (a_all >= 0 && c_best <= kK1Bins)
            for (int b = b0; b < b0 + PER; ++b)
                if (b >= a_all && b < c_best) m += (double)__ldcg(hist + b);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
        if (lane == 0) {
            const bool ok = a_all >= 0 && a_all < kK1Bins && c_best <= kK1Bins && m <= (double)kCandCap;
            sh_i[0] = ok ? 1 : 0;
            if (ok) {
                *lo_out = hist_edge(hbase, a_all);
                *hi_out = hist_edge(hbase, c_best);
                *m_out = m;
            }
        }
    }
    __syncthreads();
    return sh_i[0];
}



// Records tau of this iteration and places the window of the next one around
// the linear extrapolation of the last two thresholds.  After a window hit the
// half-width covers twice the last change of the step plus a tenth of the step
// (the extrapolation error of a smoothly converging sequence); after a miss,
// twice the step itself.  Either is capped so that about kCandTarget
// candidates are expected (density measured at the last window).  `hit`: tau
// came from K1's window.  Thread 0 only.
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
    const double center = tau_new + d1;
    double hw;
    if (!trend) {
        hw = 1e-3 * tau_new;
    } else if (hit && c.have_prev2 && c.tau_prev2 > 0.0) {
        const double d0 = c.tau_prev - c.tau_prev2;
        hw = 2.0 * fabs(d1 - d0) + 0.1 * fabs(d1) + 1e-7 * tau_new;
    } else {
        hw = 2.0 * fabs(d1) + 1e-7 * tau_new;
    }
    if (c.dens > 0.0) hw = fmin(hw, 0.5 * kCandTarget / c.dens);
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
