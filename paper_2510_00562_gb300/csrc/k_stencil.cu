// K1: the fused stencil pass of one P-PDS iteration (Algorithm 1).
//
// One CTA owns a TY x TX spatial tile and a contiguous run of bands
// [b0, b1).  It marches over the bands in order and, for each band b, in one
// pass over shared memory:
//   * u step (Eq. 21 box clamp) and its extrapolation u' = 2u+ - u for band
//     b+1, from D^T y1 + D_s^T D^T y2 + y4 (D_s^T needs D^T y2 of two bands,
//     kept from the previous step);
//   * w1, w2 steps: L y at the three grids (Condat's interpolators), the
//     group soft-threshold of Eq. 24, and w' = 2w+ - w, on the tile plus a
//     one-pixel ring (the ring is recomputed by the neighbours too, so L^T w'
//     needs no exchange);
//   * the dual ascent y1+ = y1 + g (D u' - L^T w1'), y2+ = y2 + g (D D_s u' -
//     L^T w2') for band b (y3, y4 need the l1 thresholds and come in K2);
//   * the statistics of the windowed l1-threshold search on
//     s~ = s - g_s y4 and t~ = t - g_t (D_v^T y3 + y4).
// The halo comes from the same cube loads (rows i0-2 .. i0+TY+1), so the
// tile needs y at distance 2 and w, u at distance 1.
#include <algorithm>

#include "gsstv_internal.cuh"
#include "gsstv_l1.cuh"

namespace gsstv {
namespace {

constexpr int TY = 16, TX = 32, NT = 256;
constexpr int SW = TX + 8;          // shared row width of loaded planes (origin column j0-4)
constexpr int YR = TY + 4;          // rows of y planes (origin row i0-2)
constexpr int WR = TY + 2;          // rows of w planes (origin row i0-1)
constexpr int UR = TY + 1;          // rows of u and q planes (origin row i0)
constexpr int UC = TX + 1;          // columns of the computed u' and D^T y2 (origin j0)
constexpr int Y_PL = YR * SW;
constexpr int W_PL = WR * SW;
constexpr int U_PL = UR * SW;
constexpr int C_PL = UR * UC;
constexpr int SMEM_FLOATS = 2 * 4 * Y_PL + 12 * W_PL + U_PL + 2 * U_PL + 2 * C_PL + C_PL;
constexpr int QUADS = SW / 4;
constexpr int NU = TY * TX + (TX + 1) + TY;                 // u' items: tile + bottom row + right column
constexpr int NW = TY * TX + 2 * (TX + 2) + 2 * TY;         // w' items: tile + one-pixel ring
static_assert(TY * TX % NT == 0, "tile must be a multiple of the block");

template <typename T> struct Quad;
template <> struct Quad<float> {
    static __device__ __forceinline__ float4 ld(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
};
template <> struct Quad<__nv_bfloat16> {
    static __device__ __forceinline__ float4 ld(const __nv_bfloat16* p) {
        uint2 r = __ldg(reinterpret_cast<const uint2*>(p));
        __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162*>(&r.x);
        __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162*>(&r.y);
        float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
        return make_float4(fa.x, fa.y, fb.x, fb.y);
    }
};
template <> struct Quad<__half> {
    static __device__ __forceinline__ float4 ld(const __half* p) {
        uint2 r = __ldg(reinterpret_cast<const uint2*>(p));
        __half2 a = *reinterpret_cast<__half2*>(&r.x);
        __half2 b = *reinterpret_cast<__half2*>(&r.y);
        float2 fa = __half22float2(a), fb = __half22float2(b);
        return make_float4(fa.x, fa.y, fb.x, fb.y);
    }
};

// Loads `rows` rows of one band plane (global rows row0..) and the columns
// j0-4 .. j0+TX+3 into dst (rows x SW floats); zero outside the cube.
template <typename T>
__device__ __forceinline__ void load_plane(float* dst, int rows, int row0, const T* plane,
                                           const Geom& g, int j0) {
    for (int e = threadIdx.x; e < rows * QUADS; e += NT) {
        const int r = e / QUADS, qd = e - r * QUADS;
        const int gi = row0 + r, gj = j0 - 4 + 4 * qd;
        float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gi >= 0 && gi < g.n1 && gj >= 0 && gj < g.p2)
            val = Quad<T>::ld(plane + (long long)gi * g.p2 + gj);
        *reinterpret_cast<float4*>(dst + r * SW + 4 * qd) = val;
    }
}

template <typename T>
struct K1Args {
    Geom g;
    const T *u, *s, *t, *y3, *q, *w1, *w2, *y1, *y2;
    T *u_n, *w1_n, *w2_n, *y1_n, *y2_n;
    IterParams p;
    Scal* sc;
    L1Work l1;
    int chunk;     // bands per CTA
};

template <typename T>
__global__ void __launch_bounds__(NT, 2) k1_stencil(const K1Args<T> a) {
    extern __shared__ __align__(16) float smem[];
    float* ys = smem;                       // [2 slots][4 planes][YR][SW]
    float* ws = ys + 2 * 4 * Y_PL;          // [12][WR][SW]   w then w'
    float* us = ws + 12 * W_PL;             // [UR][SW]       u of band b+1
    float* qs = us + U_PL;                  // [2 slots][UR][SW]
    float* up = qs + 2 * U_PL;              // [2 slots][UR][UC] u'
    float* gs = up + 2 * C_PL;              // [UR][UC] D^T y2 of the previous band

    __shared__ double red_d[64];
    __shared__ unsigned long long red_u[64];
    __shared__ int is_last;

    const Geom g = a.g;
    const IterParams& P = a.p;
    const int i0 = blockIdx.y * TY, j0 = blockIdx.x * TX;
    const int b0 = blockIdx.z * a.chunk;
    const int b1 = min(g.n3, b0 + a.chunk);
    const int tid = threadIdx.x;
    const long long cube = g.cube;
    const long long plane = (long long)g.n1 * g.p2;
    const float cs = (float)(1.0 - a.sc->c[P.parity]);   // y4 = (1 - c) q
    const unsigned it32 = (unsigned)a.sc->iter;           // seeds the 16-bit rounding streams

    // window of the l1 search for s (v = 0) and t (v = 1)
    const bool win_s = !P.tau_exact && a.sc->radius[0] > 0.0 && a.sc->ctl[0].window_ok;
    const bool win_t = !P.tau_exact && a.sc->radius[1] > 0.0 && a.sc->ctl[1].window_ok;
    const float lo_s = a.sc->ctl[0].theta_lo, hi_s = a.sc->ctl[0].theta_hi;
    const float lo_t = a.sc->ctl[1].theta_lo, hi_t = a.sc->ctl[1].theta_hi;
    WinAcc acc_s, acc_t;

    auto Yp = [&](int slot, int pl) { return ys + (slot * 4 + pl) * Y_PL; };

    auto load_y = [&](int band, int slot, int first_plane) {
        const T* srcs[4] = {a.y1, a.y1 + cube, a.y2, a.y2 + cube};
        for (int pl = first_plane; pl < 4; ++pl)
            load_plane<T>(Yp(slot, pl), YR, i0 - 2, srcs[pl] + band * plane, g, j0);
    };
    auto load_uq = [&](int band) {
        load_plane<T>(us, UR, i0, a.u + band * plane, g, j0);
        load_plane<T>(qs + (band & 1) * U_PL, UR, i0, a.q + band * plane, g, j0);
    };
    auto load_w = [&](int band) {
        for (int k = 0; k < 6; ++k) {
            load_plane<T>(ws + k * W_PL, WR, i0 - 1, a.w1 + k * cube + band * plane, g, j0);
            load_plane<T>(ws + (6 + k) * W_PL, WR, i0 - 1, a.w2 + k * cube + band * plane, g, j0);
        }
    };
    // D^T y = D_v^T y_v + D_h^T y_h at tile-relative (r, c) from a y slot
    auto dty = [&](int slot, int pv, int r, int c, int gi, int gj) {
        const float* yv = Yp(slot, pv);
        const float* yh = Yp(slot, pv + 1);
        const int k = (r + 2) * SW + (c + 4);
        float d = 0.f;
        if (gi >= 1) d += yv[k - SW];
        if (gi <= g.n1 - 2) d -= yv[k];
        if (gj >= 1) d += yh[k - 1];
        if (gj <= g.n2 - 2) d -= yh[k];
        return d;
    };
    // u step and u' for band bb at (r, c) in [0, TY] x [0, TX]
    auto u_item = [&](int bb, int r, int c, bool store) {
        const int gi = i0 + r, gj = j0 + c;
        const int kc = r * UC + c;
        if (gi >= g.n1 || gj >= g.n2) { up[(bb & 1) * C_PL + kc] = 0.f; gs[kc] = 0.f; return; }
        const int slot = bb & 1;
        const float d1 = dty(slot, 0, r, c, gi, gj);
        const float gcur = dty(slot, 2, r, c, gi, gj);
        float dst = 0.f;
        if (bb >= 1) dst += gs[kc];
        if (bb <= g.n3 - 2) dst -= gcur;
        const int ku = r * SW + (c + 4);
        const float y4 = cs * qs[slot * U_PL + ku];
        const float u = us[ku];
        const float un = fminf(fmaxf(u - P.gamma_u * (d1 + dst + y4), P.mu_lo), P.mu_hi);
        up[slot * C_PL + kc] = 2.f * un - u;
        gs[kc] = gcur;
        if (store && r < TY && c < TX) {
            const long long o = g.at(bb, gi, gj);
            SRStream sr((unsigned)o, it32, 2u);
            stS(a.u_n + o, un, sr);
        }
    };
    // w steps at (r, c) in [-1, TY] x [-1, TX], band b
    auto w_item = [&](int b, int r, int c) {
        const int gi = i0 + r, gj = j0 + c;
        const int kw = (r + 1) * SW + (c + 4);
        if (gi < 0 || gi >= g.n1 || gj < 0 || gj >= g.n2) {
#pragma unroll
            for (int k = 0; k < 12; ++k) ws[k * W_PL + kw] = 0.f;
            return;
        }
        const bool mv = gi < g.n1 - 1, mh = gj < g.n2 - 1;
        const bool inner = r >= 0 && r < TY && c >= 0 && c < TX;
        const int slot = b & 1;
        const int ky = (r + 2) * SW + (c + 4);
#pragma unroll
        for (int set = 0; set < 2; ++set) {
            const float* yv = Yp(slot, 2 * set);
            const float* yh = Yp(slot, 2 * set + 1);
            // y_v masked on the last row, y_h on the last column (where D is 0)
            auto V = [&](int dr, int dc) { return (gi + dr == g.n1 - 1) ? 0.f : yv[ky + dr * SW + dc]; };
            auto H = [&](int dr, int dc) { return (gj + dc == g.n2 - 1) ? 0.f : yh[ky + dr * SW + dc]; };
            const float v00 = V(0, 0), vm0 = V(-1, 0), v01 = V(0, 1), vm1 = V(-1, 1);
            const float h00 = H(0, 0), h0m = H(0, -1), h10 = H(1, 0), h1m = H(1, -1);
            float Lv[3], Lh[3];
            Lv[0] = mv ? v00 : 0.f;
            Lh[0] = mv ? 0.25f * (h00 + h0m + h10 + h1m) : 0.f;
            Lv[1] = mh ? 0.25f * (v00 + vm0 + v01 + vm1) : 0.f;
            Lh[1] = mh ? h00 : 0.f;
            Lv[2] = 0.5f * (v00 + vm0);
            Lh[2] = 0.5f * (h00 + h0m);
            const float gam = set ? P.gamma_w2 : P.gamma_w1;
            const float thr = set ? P.thr_w2 : P.thr_w1;
            T* dst = set ? a.w2_n : a.w1_n;
            SRStream sr((unsigned)g.at(b, gi, gj), it32, 4u + set);
#pragma unroll
            for (int gr = 0; gr < 3; ++gr) {
                float* pv = ws + (6 * set + 2 * gr) * W_PL + kw;
                float* ph = pv + W_PL;
                const float wv = *pv, wh = *ph;
                const float xv = wv + gam * Lv[gr], xh = wh + gam * Lh[gr];
                const float n = sqrtf(xv * xv + xh * xh);
                const float sc = n > thr ? 1.f - thr / n : 0.f;
                const float nv = sc * xv, nh = sc * xh;
                *pv = 2.f * nv - wv;
                *ph = 2.f * nh - wh;
                if (inner) {
                    const long long o = g.at(b, gi, gj);
                    stS(dst + (2 * gr) * cube + o, nv, sr);
                    stS(dst + (2 * gr + 1) * cube + o, nh, sr);
                }
            }
        }
    };
    auto u_ring = [&](int k, int& r, int& c) {
        if (k < TY * TX) { r = k / TX; c = k - r * TX; return; }
        k -= TY * TX;
        if (k < TX + 1) { r = TY; c = k; return; }
        r = k - (TX + 1); c = TX;
    };
    auto w_ring = [&](int k, int& r, int& c) {
        if (k < TY * TX) { r = k / TX; c = k - r * TX; return; }
        k -= TY * TX;
        if (k < TX + 2) { r = -1; c = k - 1; return; }
        k -= TX + 2;
        if (k < TX + 2) { r = TY; c = k - 1; return; }
        k -= TX + 2;
        if (k < TY) { r = k; c = -1; return; }
        r = k - TY; c = TX;
    };

    // ---- prologue: D^T y2 of band b0-1 and u' of band b0 ----
    if (b0 >= 1) {
        load_y(b0 - 1, (b0 - 1) & 1, 2);
        __syncthreads();
        for (int e = tid; e < UR * UC; e += NT) {
            const int r = e / UC, c = e - r * UC;
            const int gi = i0 + r, gj = j0 + c;
            gs[e] = (gi < g.n1 && gj < g.n2) ? dty((b0 - 1) & 1, 2, r, c, gi, gj) : 0.f;
        }
    }
    load_y(b0, b0 & 1, 0);
    load_uq(b0);
    __syncthreads();
    for (int e = tid; e < NU; e += NT) {
        int r, c;
        u_ring(e, r, c);
        u_item(b0, r, c, true);
    }
    __syncthreads();

    // ---- band march ----
    for (int b = b0; b < b1; ++b) {
        const bool has_next = b + 1 < g.n3;
        if (has_next) {
            load_y(b + 1, (b + 1) & 1, 0);
            load_uq(b + 1);
        }
        load_w(b);
        __syncthreads();
        for (int e = tid; e < NU + NW; e += NT) {
            int r, c;
            if (e < NU) {
                if (has_next) { u_ring(e, r, c); u_item(b + 1, r, c, b + 1 < b1); }
            } else {
                w_ring(e - NU, r, c);
                w_item(b, r, c);
            }
        }
        __syncthreads();
        const float* upb = up + (b & 1) * C_PL;
        const float* upn = up + ((b + 1) & 1) * C_PL;
        const long long bo = (long long)b * plane;
        for (int e = tid; e < TY * TX; e += NT) {
            const int r = e / TX, c = e - r * TX;
            const int gi = i0 + r, gj = j0 + c;
            const bool valid = gi < g.n1 && gj < g.n2;
            float xs = 0.f, xt = 0.f;
            if (valid) {
                const int kc = r * UC + c;
                const float u0 = upb[kc];
                const bool mv = gi < g.n1 - 1, mh = gj < g.n2 - 1;
                const float duv = mv ? upb[kc + UC] - u0 : 0.f;
                const float duh = mh ? upb[kc + 1] - u0 : 0.f;
                float ddv = 0.f, ddh = 0.f;
                if (has_next) {
                    const float d0 = upn[kc] - u0;
                    if (mv) ddv = (upn[kc + UC] - upb[kc + UC]) - d0;
                    if (mh) ddh = (upn[kc + 1] - upb[kc + 1]) - d0;
                }
                const int kw = (r + 1) * SW + (c + 4);
                float gv[2], gh[2];
#pragma unroll
                for (int set = 0; set < 2; ++set) {
                    const float* W = ws + 6 * set * W_PL + kw;
                    auto Wk = [&](int k, int dr, int dc) { return W[k * W_PL + dr * SW + dc]; };
                    // a = grid 0 horizontal (masked by its row), bb = grid 1 vertical (masked by its column)
                    auto A_ = [&](int dr, int dc) { return (gi + dr < g.n1 - 1) ? Wk(1, dr, dc) : 0.f; };
                    auto B_ = [&](int dr, int dc) { return (gj + dc < g.n2 - 1) ? Wk(2, dr, dc) : 0.f; };
                    gv[set] = mv ? (Wk(0, 0, 0) + 0.25f * (B_(0, 0) + B_(1, 0) + B_(0, -1) + B_(1, -1))
                                    + 0.5f * (Wk(4, 0, 0) + Wk(4, 1, 0)))
                                 : 0.f;
                    gh[set] = mh ? (0.25f * (A_(0, 0) + A_(0, 1) + A_(-1, 0) + A_(-1, 1)) + Wk(3, 0, 0)
                                    + 0.5f * (Wk(5, 0, 0) + Wk(5, 0, 1)))
                                 : 0.f;
                }
                const int ky = (r + 2) * SW + (c + 4);
                const int slot = b & 1;
                const long long o = g.at(b, gi, gj);
                SRStream sr((unsigned)o, it32, 3u);
                stS(a.y1_n + o, Yp(slot, 0)[ky] + P.gamma_y1 * (duv - gv[0]), sr);
                stS(a.y1_n + cube + o, Yp(slot, 1)[ky] + P.gamma_y1 * (duh - gh[0]), sr);
                stS(a.y2_n + o, Yp(slot, 2)[ky] + P.gamma_y2 * (ddv - gv[1]), sr);
                stS(a.y2_n + cube + o, Yp(slot, 3)[ky] + P.gamma_y2 * (ddh - gh[1]), sr);
                if (win_s || win_t) {
                    const float qv = qs[slot * U_PL + r * SW + (c + 4)];
                    const long long oi = bo + (long long)gi * g.p2 + gj;
                    const float sv = ldT(a.s + oi), tv = ldT(a.t + oi), y3v = ldT(a.y3 + oi);
                    const float y3u = gi >= 1 ? ldT(a.y3 + oi - g.p2) : 0.f;
                    s_t_tilde(sv, tv, y3v, y3u, qv, cs, gi, g.n1, P.gamma_s, P.gamma_t, xs, xt);
                }
            }
            if (win_s) {
                const float x = fabsf(xs);
                const bool hi = valid && x > hi_s;
                if (hi) { acc_s.n++; acc_s.s.add(x); }
                append_candidate(valid && !hi && x > lo_s, x, a.l1.cand[0], &a.sc->acc[0].m);
            }
            if (win_t) {
                const float x = fabsf(xt);
                const bool hi = valid && x > hi_t;
                if (hi) { acc_t.n++; acc_t.s.add(x); }
                append_candidate(valid && !hi && x > lo_t, x, a.l1.cand[1], &a.sc->acc[1].m);
            }
        }
        __syncthreads();
    }

    // ---- window statistics of this CTA, then the last CTA finishes tau ----
    const int cta = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int ncta = gridDim.x * gridDim.y * gridDim.z;
    if (win_s || win_t) {
        const unsigned long long ns = block_sum(acc_s.n, red_u);
        const double ss = block_sum(acc_s.s.value(), red_d);
        const unsigned long long nt = block_sum(acc_t.n, red_u);
        const double st = block_sum(acc_t.s.value(), red_d);
        if (tid == 0) {
            a.l1.k1_n[2 * cta] = ns;
            a.l1.k1_n[2 * cta + 1] = nt;
            a.l1.k1_s[2 * cta] = ss;
            a.l1.k1_s[2 * cta + 1] = st;
        }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) is_last = (atomicAdd(&a.sc->k1_ticket, 1u) == (unsigned)(ncta - 1));
    __syncthreads();
    if (!is_last) return;
    __threadfence();

    for (int v = 0; v < 2; ++v) {
        L1Ctl& C = a.sc->ctl[v];
        const double r = a.sc->radius[v];
        const bool win = v == 0 ? win_s : win_t;
        if (!(r > 0.0)) {
            if (tid == 0) {
                C.tau = __int_as_float(0x7f800000);  // +inf: the ball is {0}
                C.have_tau = 1;
                C.need = NEED_NONE;
                C.window_ok = 0;
            }
            continue;
        }
        if (!win) {
            if (tid == 0) {
                C.need = NEED_RADIX0; C.prefix = 0; C.n_above = 0; C.s_above = 0.0; C.exact_runs++;
            }
            continue;
        }
        unsigned long long n = 0;
        double s = 0.0;
        for (int k = tid; k < ncta; k += NT) {
            n += __ldcg(a.l1.k1_n + 2 * k + v);
            s += __ldcg(a.l1.k1_s + 2 * k + v);
        }
        n = block_sum(n, red_u);
        s = block_sum(s, red_d);
        const unsigned m = __ldcg(&a.sc->acc[v].m);
        const double tlo = C.theta_lo, thi = C.theta_hi;
        double tau = 0.0;
        WinInfo wi;
        const int miss = l1_window_finish((double)n, s, a.l1.cand[v], m, tlo, thi, r, &tau, red_d, red_u, &wi);
        if (tid == 0) {
            if (!miss) {
                l1_record_tau(C, tau, (double)min(m, kCandCap), thi - tlo, true);
                C.hits++;
            } else {
                l1_after_miss(C, miss, wi, (double)n, m, tlo, thi);
            }
            a.sc->acc[v].m = 0;
        }
        __syncthreads();
    }
    if (tid == 0) a.sc->k1_ticket = 0;
}

template <typename T>
int launch_k1_t(const Geom& g, const IterBufs& b, const IterParams& p, Scal* sc, const L1Work& w,
                cudaStream_t st) {
    const size_t smem = SMEM_FLOATS * sizeof(float);
    K1Args<T> a;
    a.g = g;
    a.u = (const T*)b.u; a.s = (const T*)b.s; a.t = (const T*)b.t; a.y3 = (const T*)b.y3;
    a.q = (const T*)b.q; a.w1 = (const T*)b.w1; a.w2 = (const T*)b.w2;
    a.y1 = (const T*)b.y1; a.y2 = (const T*)b.y2;
    a.u_n = (T*)b.u_n; a.w1_n = (T*)b.w1_n; a.w2_n = (T*)b.w2_n; a.y1_n = (T*)b.y1_n; a.y2_n = (T*)b.y2_n;
    a.p = p;
    a.sc = sc;
    a.l1 = w;
    const int tiles = ((g.n2 + TX - 1) / TX) * ((g.n1 + TY - 1) / TY);
    const int target = device_sms() * 16;                  // about 16 CTAs per SM
    int chunks = (target + tiles - 1) / tiles;
    chunks = max(1, min(chunks, (g.n3 + 7) / 8));          // at least 8 bands per CTA
    a.chunk = (g.n3 + chunks - 1) / chunks;
    chunks = (g.n3 + a.chunk - 1) / a.chunk;
    dim3 grid((g.n2 + TX - 1) / TX, (g.n1 + TY - 1) / TY, chunks);
    k1_stencil<T><<<grid, NT, smem, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace

int k1_configure(int storage) {
    const int smem = SMEM_FLOATS * sizeof(float);
    cudaError_t e = cudaErrorInvalidValue;
    switch (storage) {
        case 0: e = cudaFuncSetAttribute(k1_stencil<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); break;
        case 1: e = cudaFuncSetAttribute(k1_stencil<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); break;
        case 2: e = cudaFuncSetAttribute(k1_stencil<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); break;
    }
    return e == cudaSuccess ? 0 : -3;
}

int k1_grid_ctas(const Geom& g) {
    const int tiles = ((g.n2 + TX - 1) / TX) * ((g.n1 + TY - 1) / TY);
    const int target = device_sms() * 16;
    int chunks = (target + tiles - 1) / tiles;
    chunks = std::max(1, std::min(chunks, (g.n3 + 7) / 8));
    const int chunk = (g.n3 + chunks - 1) / chunks;
    chunks = (g.n3 + chunk - 1) / chunk;
    return tiles * chunks;
}

int launch_k1(int storage, const Geom& g, const IterBufs& b, const IterParams& p, Scal* sc,
              const L1Work& w, int, cudaStream_t st) {
    switch (storage) {
        case 0: return launch_k1_t<float>(g, b, p, sc, w, st);
        case 1: return launch_k1_t<__nv_bfloat16>(g, b, p, sc, w, st);
        case 2: return launch_k1_t<__half>(g, b, p, sc, w, st);
    }
    return -1;
}

}  // namespace gsstv
