// K1, TMA-fed: the fused stencil pass of one P-PDS iteration (Algorithm 1).
//
// Same arithmetic as the cooperative-load kernel in k_stencil.cu (u step and
// u' for band b+1; w1, w2 group soft-thresholds and w' on the tile plus a
// one-pixel ring; y1, y2 ascent for band b; window statistics of the l1
// threshold search), fed differently: each band's planes are brought into
// shared memory by bulk tensor (TMA) copies that one thread issues two bands
// ahead, completing on mbarriers, so the loads of band b+2 (y, u, q, s, t,
// y3) and b+1 (w) are in flight while band b computes.  One CTA of 512
// threads per SM owns a 16 x 32 tile and a run of bands.  Tiles whose halo
// stays off the image border take a specialised path with no boundary masks.
//
// The two compute phases are software-pipelined over the bands: while the w
// steps and u' of band b run, the dual ascent and the l1 statistics of band
// b-1 (which only read what the previous step completed) run beside them, so
// each band costs one CTA barrier.  Shared memory per CTA (FP32): 4 slots of the
// y-group (4 y planes with a 2-pixel halo, u and q with a 1-pixel halo
// below/right, s, t, y3 with one row above), 3 slots of the 12 w planes
// (1-pixel halo), u' of three bands and D^T y2 of the previous band: about
// 211 KB.
#include <algorithm>
#include <type_traits>

#include "gsstv_internal.cuh"
#include "gsstv_l1.cuh"
#include "gsstv_tma.cuh"

namespace gsstv {

// ---------------------------------------------------------------------------
// host: tensor maps
// ---------------------------------------------------------------------------
namespace {
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeFn encode_fn() {
    static EncodeFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    }
    return fn;
}
}  // namespace

int tma_encode_cubes(CUtensorMap* map, const void* base, int elem_bytes, int n1, int n2, int n3, int p2,
                     int ncubes, int box_x, int box_y) {
    EncodeFn fn = encode_fn();
    if (!fn) return -3;
    const CUtensorMapDataType dt = elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                   : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;  // 16-bit: bits only
    cuuint64_t dims[3] = {(cuuint64_t)n2, (cuuint64_t)n1, (cuuint64_t)n3 * (cuuint64_t)ncubes};
    cuuint64_t strides[2] = {(cuuint64_t)p2 * elem_bytes, (cuuint64_t)p2 * elem_bytes * n1};
    cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1u};
    cuuint32_t estr[3] = {1u, 1u, 1u};
    const CUresult r = fn(map, dt, 3, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -3;
}

namespace {

template <typename T>
struct Lay {
    static constexpr int TY = 16, TX = 32, NT = 512;
    static constexpr int ES = sizeof(T);
    static constexpr int OX = 16 / ES;             // left halo columns: boxes start 16-byte aligned
    static constexpr int SW = TX + 2 * OX;         // width of the staged planes
    static constexpr int YR = TY + 4, WR = TY + 2, UR = TY + 1, UC = TX + 1;
    static constexpr int WPC = TX + 2;             // width of the separate w' planes (16-bit storage)
    static constexpr int pad(int b) { return (b + 127) / 128 * 128; }
    static constexpr int Y_B = pad(YR * SW * ES);
    static constexpr int W_B = pad(WR * SW * ES);
    static constexpr int U_B = pad(UR * SW * ES);
    static constexpr int S_B = pad(TY * TX * ES);
    static constexpr int Y3_B = pad((TY + 1) * TX * ES);
    static constexpr int YG_B = 4 * Y_B + 2 * U_B + 2 * S_B + Y3_B;
    static constexpr int WG_B = 12 * W_B;
    static constexpr bool kInPlace = ES == 4;      // w' overwrites the staged w planes
    static constexpr int NYS = 4, NWS = 3, NUS = 3;  // ring depths: y-group, w, u'
    static constexpr int WP1_B = pad(12 * WR * WPC * 4);
    static constexpr int WP_B = kInPlace ? 0 : 2 * WP1_B;
    static constexpr int UP1 = UR * UC;              // floats of one u' plane
    static constexpr int UP_B = pad(NUS * UP1 * 4);
    static constexpr int G_B = pad(UR * UC * 4);
    static constexpr int OFF_WG = NYS * YG_B;
    static constexpr int OFF_WP = OFF_WG + NWS * WG_B;
    static constexpr int OFF_UP = OFF_WP + WP_B;
    static constexpr int OFF_G = OFF_UP + UP_B;
    static constexpr int OFF_BAR = OFF_G + G_B;
    static constexpr int SMEM = OFF_BAR + (NYS + NWS) * 8;
    // offsets inside a y-group slot
    static constexpr int O_U = 4 * Y_B, O_Q = O_U + U_B, O_S = O_Q + U_B, O_T = O_S + S_B, O_Y3 = O_T + S_B;
    // bytes each group's copies deliver
    static constexpr unsigned YG_TX = 4u * YR * SW * ES + 2u * UR * SW * ES + 2u * TY * TX * ES + (TY + 1u) * TX * ES;
    static constexpr unsigned WG_TX = 12u * WR * SW * ES;
    static constexpr int NU = TY * TX + (TX + 1) + TY;
    static constexpr int NW = TY * TX + 2 * (TX + 2) + 2 * TY;
    static_assert(TY * TX == NT, "one tile voxel per thread");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

template <typename T>
struct K1TArgs {
    Geom g;
    T *u_n, *w1_n, *w2_n, *y1_n, *y2_n;
    IterParams p;
    Scal* sc;
    L1Work l1;
    int chunk;
};

template <typename T> __device__ __forceinline__ float sld(const T* p) { return ldT(p); }

// Per-CTA running state shared by the two tile paths.
struct K1State {
    WinAcc acc_s, acc_t;
    unsigned n_y = 0, n_w = 0;   // groups issued so far (thread 0 only)
};

template <typename T, bool EDGE>
__device__ __forceinline__ bool k1_tile(const K1Maps& M, const K1TArgs<T>& a, unsigned char* sm, int i0,
                                        int j0, int b0, int b1, K1State& S, bool win_s, bool win_t,
                                        float lo_s, float hi_s, float lo_t, float hi_t, float cs) {
    using L = Lay<T>;
    constexpr int TY = L::TY, TX = L::TX, SW = L::SW, OX = L::OX, UC = L::UC;
    constexpr int WP_ROW = L::kInPlace ? SW : L::WPC;
    const Geom& g = a.g;
    const IterParams& P = a.p;
    const int tid = threadIdx.x;
    const unsigned cube = (unsigned)g.cube;        // < 2^31 (checked at handle creation)
    const unsigned plane = (unsigned)g.n1 * (unsigned)g.p2;
    uint64_t* ybar = reinterpret_cast<uint64_t*>(sm + L::OFF_BAR);
    uint64_t* wbar = ybar + L::NYS;
    float* up = reinterpret_cast<float*>(sm + L::OFF_UP);
    float* gs = reinterpret_cast<float*>(sm + L::OFF_G);
    const int bstart = max(b0 - 1, 0);
    const int blast = min(b1, g.n3 - 1);
    const unsigned it32 = (unsigned)a.sc->iter;     // seeds the 16-bit rounding streams

    // ---- ring slots (computed once per band by the callers below) ----
    auto yg = [&](int band) { return sm + ((band - bstart) % L::NYS) * L::YG_B; };
    auto wg = [&](int band) { return sm + L::OFF_WG + ((band - b0) % L::NWS) * L::WG_B; };
    // w' of a band: in place in its w slot (FP32), else in one of two float
    // planes that alternate with the band (16-bit storage)
    auto wpl = [&](int band) -> float* {
        if constexpr (L::kInPlace) return reinterpret_cast<float*>(wg(band));
        else return reinterpret_cast<float*>(sm + L::OFF_WP + ((band - b0) & 1) * L::WP1_B);
    };
    constexpr int WP_PL = L::kInPlace ? L::W_B / 4 : L::WR * L::WPC;   // floats between w' planes
    auto upl = [&](int band) { return up + (band % L::NUS) * L::UP1; };
    auto wp_idx = [&](int r, int c) {
        if constexpr (L::kInPlace) return (r + 1) * SW + (c + OX);
        else return (r + 1) * L::WPC + (c + 1);
    };

    auto issue_y = [&](int band) {
        unsigned char* s = yg(band);
        uint64_t* bar = ybar + (band - bstart) % L::NYS;
        mbar_arrive_expect_tx(bar, L::YG_TX);
        tma_load_3d(s + 0 * L::Y_B, &M.y1, j0 - OX, i0 - 2, band, bar);
        tma_load_3d(s + 1 * L::Y_B, &M.y1, j0 - OX, i0 - 2, g.n3 + band, bar);
        tma_load_3d(s + 2 * L::Y_B, &M.y2, j0 - OX, i0 - 2, band, bar);
        tma_load_3d(s + 3 * L::Y_B, &M.y2, j0 - OX, i0 - 2, g.n3 + band, bar);
        tma_load_3d(s + L::O_U, &M.u, j0 - OX, i0, band, bar);
        tma_load_3d(s + L::O_Q, &M.q, j0 - OX, i0, band, bar);
        tma_load_3d(s + L::O_S, &M.s, j0, i0, band, bar);
        tma_load_3d(s + L::O_T, &M.t, j0, i0, band, bar);
        tma_load_3d(s + L::O_Y3, &M.y3, j0, i0 - 1, band, bar);
        S.n_y++;
    };
    auto issue_w = [&](int band) {
        unsigned char* s = wg(band);
        uint64_t* bar = wbar + (band - b0) % L::NWS;
        mbar_arrive_expect_tx(bar, L::WG_TX);
        for (int k = 0; k < 6; ++k) tma_load_3d(s + k * L::W_B, &M.w1, j0 - OX, i0 - 1, k * g.n3 + band, bar);
        for (int k = 0; k < 6; ++k) tma_load_3d(s + (6 + k) * L::W_B, &M.w2, j0 - OX, i0 - 1, k * g.n3 + band, bar);
        S.n_w++;
    };
    auto wait_y = [&](int band) {
        return mbar_wait(ybar + (band - bstart) % L::NYS, ((band - bstart) / L::NYS) & 1);
    };
    auto wait_w = [&](int band) { return mbar_wait(wbar + (band - b0) % L::NWS, ((band - b0) / L::NWS) & 1); };

    // D^T y = D_v^T y_v + D_h^T y_h at tile-relative (r, c); yv, yh: y planes
    auto dty = [&](const T* yv, const T* yh, int r, int c) {
        const int k = (r + 2) * SW + (c + OX);
        if constexpr (EDGE) {
            const int gi = i0 + r, gj = j0 + c;
            float d = 0.f;
            if (gi >= 1) d += sld(yv + k - SW);
            if (gi <= g.n1 - 2) d -= sld(yv + k);
            if (gj >= 1) d += sld(yh + k - 1);
            if (gj <= g.n2 - 2) d -= sld(yh + k);
            return d;
        } else {
            return ((sld(yv + k - SW) - sld(yv + k)) + sld(yh + k - 1)) - sld(yh + k);
        }
    };
    // u step and u' of band bb at (r, c) in [0, TY] x [0, TX]; ys: y-group of
    // bb; upb: u' plane of bb; dst: u+ of this voxel, or null (no store)
    auto u_item = [&](const unsigned char* ys, float* upb, int bb, int r, int c, T* dst) {
        const int kc = r * UC + c;
        if constexpr (EDGE) {
            if (i0 + r >= g.n1 || j0 + c >= g.n2) { upb[kc] = 0.f; gs[kc] = 0.f; return; }
        }
        const T* yp = reinterpret_cast<const T*>(ys);
        const float d1 = dty(yp, yp + L::Y_B / L::ES, r, c);
        const float gcur = dty(yp + 2 * (L::Y_B / L::ES), yp + 3 * (L::Y_B / L::ES), r, c);
        float dst_ = 0.f;
        if (bb >= 1) dst_ += gs[kc];
        if (bb <= g.n3 - 2) dst_ -= gcur;
        const int ku = r * SW + (c + OX);
        const float y4 = cs * sld(reinterpret_cast<const T*>(ys + L::O_Q) + ku);
        const float u = sld(reinterpret_cast<const T*>(ys + L::O_U) + ku);
        const float un = fminf(fmaxf(u - P.gamma_u * (d1 + dst_ + y4), P.mu_lo), P.mu_hi);
        upb[kc] = 2.f * un - u;
        gs[kc] = gcur;
        if (dst) {
            SRStream sr((unsigned)(dst - a.u_n), it32, 2u);
            stS(dst, un, sr);
        }
    };
    // w step of one set (a compile-time constant: 0 = w1, 1 = w2) at (r, c)
    // in [-1, TY] x [-1, TX]; ys: y-group, wst: staged w planes, wp: w' planes
    // of the band; dst: w+ of this voxel (set's first plane), or null on the ring
    auto w_item = [&](auto set_c, const unsigned char* ys, const T* wst, float* wp, int r, int c, T* dst) {
        constexpr int set = decltype(set_c)::value;
        const int kw = (r + 1) * SW + (c + OX);
        const int kp = wp_idx(r, c);
        const int gi = i0 + r, gj = j0 + c;
        if constexpr (EDGE) {
            if (gi < 0 || gi >= g.n1 || gj < 0 || gj >= g.n2) {
#pragma unroll
                for (int k = 6 * set; k < 6 * set + 6; ++k) wp[k * WP_PL + kp] = 0.f;
                return;
            }
        }
        const bool mv = !EDGE || gi < g.n1 - 1, mh = !EDGE || gj < g.n2 - 1;
        const int ky = (r + 2) * SW + (c + OX);
        const T* yv = reinterpret_cast<const T*>(ys + (2 * set) * L::Y_B) + ky;
        const T* yh = reinterpret_cast<const T*>(ys + (2 * set + 1) * L::Y_B) + ky;
        auto V = [&](int dr, int dc) {
            if constexpr (EDGE) return (gi + dr == g.n1 - 1) ? 0.f : sld(yv + dr * SW + dc);
            else return sld(yv + dr * SW + dc);
        };
        auto H = [&](int dr, int dc) {
            if constexpr (EDGE) return (gj + dc == g.n2 - 1) ? 0.f : sld(yh + dr * SW + dc);
            else return sld(yh + dr * SW + dc);
        };
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
        const float thr2 = thr * thr;
        SRStream sr(dst ? (unsigned)(dst - (set ? a.w2_n : a.w1_n)) : 0u, it32, 4u + set);
#pragma unroll
        for (int gr = 0; gr < 3; ++gr) {
            const int kv = 6 * set + 2 * gr;
            const float wv = sld(wst + kv * (L::W_B / L::ES) + kw);
            const float wh = sld(wst + (kv + 1) * (L::W_B / L::ES) + kw);
            const float xv = wv + gam * Lv[gr], xh = wh + gam * Lh[gr];
            // Eq. 24: max(1 - thr / ||x||, 0) x, with 1 / ||x|| from rsqrt
            const float n2 = xv * xv + xh * xh;
            const float sc = n2 > thr2 ? fmaxf(1.f - thr * rsqrtf(n2), 0.f) : 0.f;
            const float nv = sc * xv, nh = sc * xh;
            wp[kv * WP_PL + kp] = 2.f * nv - wv;
            wp[(kv + 1) * WP_PL + kp] = 2.f * nh - wh;
            if (dst) {
                stS(dst + (2 * gr) * cube, nv, sr);
                stS(dst + (2 * gr + 1) * cube, nh, sr);
            }
        }
    };
    using Set0 = std::integral_constant<int, 0>;
    using Set1 = std::integral_constant<int, 1>;

    // ---- this thread's tile voxel and its share of the one-pixel ring ----
    const int r_t = tid / TX, c_t = tid - (tid / TX) * TX;
    const int gi_t = i0 + r_t, gj_t = j0 + c_t;
    const bool valid_t = !EDGE || (gi_t < g.n1 && gj_t < g.n2);
    const unsigned o_t = valid_t ? (unsigned)gi_t * (unsigned)g.p2 + (unsigned)gj_t : 0u;
    // ring w positions: 2 (TX + 2) + 2 TY; each set takes four warps (128
    // threads, one position each) so a warp never mixes the two sets; ring u'
    // positions ((TX + 1) + TY) go to the next warps
    constexpr int NWR = 2 * (TX + 2) + 2 * TY;
    constexpr int NUR = (TX + 1) + TY;
    static_assert(NWR <= 128 && 256 + NUR <= L::NT, "ring work layout");
    int rw_r = 0, rw_c = 0, ru_r = 0, ru_c = 0;
    const int rw_set = tid >> 7;                       // 0 or 1 for tid < 256
    const bool has_rw = tid < 256 && (tid & 127) < NWR;
    const bool has_ru = tid >= 256 && tid < 256 + NUR;
    if (has_rw) {
        int k = tid & 127;
        if (k < TX + 2) { rw_r = -1; rw_c = k - 1; }
        else if ((k -= TX + 2) < TX + 2) { rw_r = TY; rw_c = k - 1; }
        else if ((k -= TX + 2) < TY) { rw_r = k; rw_c = -1; }
        else { rw_r = k - TY; rw_c = TX; }
    }
    if (has_ru) {
        const int k = tid - 256;
        if (k < TX + 1) { ru_r = TY; ru_c = k; } else { ru_r = k - (TX + 1); ru_c = TX; }
    }

    // ---- dual ascent of y1, y2 and the l1 window statistics of one band ----
    // Reads the band's completed w', u' of the band and the next, its y-group.
    auto t_item = [&](int band) {
        const bool nxt = band + 1 < g.n3;
        const float* upb = upl(band);
        const float* upn = upl(band + 1);
        const unsigned char* ys = yg(band);
        const float* wp = wpl(band);
        const unsigned ob = (unsigned)band * plane + o_t;
        float xs = 0.f, xt = 0.f;
        if (valid_t) {
            const int r = r_t, c = c_t;
            const int kc = r * UC + c;
            const float u0 = upb[kc];
            const bool mv = !EDGE || gi_t < g.n1 - 1, mh = !EDGE || gj_t < g.n2 - 1;
            const float duv = mv ? upb[kc + UC] - u0 : 0.f;
            const float duh = mh ? upb[kc + 1] - u0 : 0.f;
            float ddv = 0.f, ddh = 0.f;
            if (nxt) {
                const float d0 = upn[kc] - u0;
                if (mv) ddv = (upn[kc + UC] - upb[kc + UC]) - d0;
                if (mh) ddh = (upn[kc + 1] - upb[kc + 1]) - d0;
            }
            const float* wk = wp + wp_idx(r, c);
            float gv[2], gh[2];
#pragma unroll
            for (int set = 0; set < 2; ++set) {
                auto Wk = [&](int k, int dr, int dc) { return wk[(6 * set + k) * WP_PL + dr * WP_ROW + dc]; };
                auto A_ = [&](int dr, int dc) {
                    if constexpr (EDGE) return (gi_t + dr < g.n1 - 1) ? Wk(1, dr, dc) : 0.f;
                    else return Wk(1, dr, dc);
                };
                auto B_ = [&](int dr, int dc) {
                    if constexpr (EDGE) return (gj_t + dc < g.n2 - 1) ? Wk(2, dr, dc) : 0.f;
                    else return Wk(2, dr, dc);
                };
                gv[set] = mv ? (Wk(0, 0, 0) + 0.25f * (B_(0, 0) + B_(1, 0) + B_(0, -1) + B_(1, -1))
                                + 0.5f * (Wk(4, 0, 0) + Wk(4, 1, 0)))
                             : 0.f;
                gh[set] = mh ? (0.25f * (A_(0, 0) + A_(0, 1) + A_(-1, 0) + A_(-1, 1)) + Wk(3, 0, 0)
                                + 0.5f * (Wk(5, 0, 0) + Wk(5, 0, 1)))
                             : 0.f;
            }
            const int ky = (r + 2) * SW + (c + OX);
            const T* yp = reinterpret_cast<const T*>(ys) + ky;
            constexpr int YPL = L::Y_B / L::ES;
            SRStream sr(ob, it32, 3u);
            stS(a.y1_n + ob, sld(yp) + P.gamma_y1 * (duv - gv[0]), sr);
            stS(a.y1_n + cube + ob, sld(yp + YPL) + P.gamma_y1 * (duh - gh[0]), sr);
            stS(a.y2_n + ob, sld(yp + 2 * YPL) + P.gamma_y2 * (ddv - gv[1]), sr);
            stS(a.y2_n + cube + ob, sld(yp + 3 * YPL) + P.gamma_y2 * (ddh - gh[1]), sr);
            if (win_s || win_t) {
                const T* q = reinterpret_cast<const T*>(ys + L::O_Q);
                const T* sp = reinterpret_cast<const T*>(ys + L::O_S);
                const T* tp = reinterpret_cast<const T*>(ys + L::O_T);
                const T* y3p = reinterpret_cast<const T*>(ys + L::O_Y3);
                const float qv = sld(q + r * SW + (c + OX));
                const float y3v = sld(y3p + (r + 1) * TX + c);
                const float y3u = (!EDGE || gi_t >= 1) ? sld(y3p + r * TX + c) : 0.f;
                s_t_tilde(sld(sp + r * TX + c), sld(tp + r * TX + c), y3v, y3u, qv, cs, gi_t, g.n1,
                          P.gamma_s, P.gamma_t, xs, xt);
            }
        }
        if (win_s) {
            const float x = fabsf(xs);
            const bool hi = valid_t && x > hi_s;
            if (hi) { S.acc_s.n++; S.acc_s.s.add(x); }
            append_candidate(valid_t && !hi && x > lo_s, x, a.l1.cand[0], &a.sc->acc[0].m);
        }
        if (win_t) {
            const float x = fabsf(xt);
            const bool hi = valid_t && x > hi_t;
            if (hi) { S.acc_t.n++; S.acc_t.s.add(x); }
            append_candidate(valid_t && !hi && x > lo_t, x, a.l1.cand[1], &a.sc->acc[1].m);
        }
    };

    // ---- prologue: D^T y2 of band b0-1 and u' of band b0 ----
    if (tid == 0) {
        for (int band = bstart; band <= min(bstart + 2, blast); ++band) issue_y(band);
        issue_w(b0);
    }
    bool ok = true;
    if (b0 >= 1) {
        ok = wait_y(b0 - 1);
        const T* yp = reinterpret_cast<const T*>(yg(b0 - 1));
        for (int e = tid; e < L::UR * UC; e += L::NT) {
            const int r = e / UC, c = e - r * UC;
            if (EDGE && (i0 + r >= g.n1 || j0 + c >= g.n2)) { gs[e] = 0.f; continue; }
            gs[e] = dty(yp + 2 * (L::Y_B / L::ES), yp + 3 * (L::Y_B / L::ES), r, c);
        }
    }
    ok = wait_y(b0) && ok;
    ok = __syncthreads_and(ok);
    if (!ok) return false;
    {
        const unsigned char* ys0 = yg(b0);
        float* up0 = upl(b0);
        u_item(ys0, up0, b0, r_t, c_t, valid_t ? a.u_n + ((unsigned)b0 * plane + o_t) : nullptr);
        if (has_ru) u_item(ys0, up0, b0, ru_r, ru_c, nullptr);
    }
    __syncthreads();

    // ---- band march, one barrier per band: w steps and u' of band b beside
    // the dual ascent of band b-1 ----
    for (int b = b0; b < b1; ++b) {
        const bool has_next = b + 1 < g.n3;
        if (tid == 0) {
            if (b + 2 <= blast && (b + 2 - bstart) >= 3) issue_y(b + 2);
            if (b + 1 < b1) issue_w(b + 1);
        }
        bool okb = wait_w(b);
        if (has_next) okb = wait_y(b + 1) && okb;
        if (okb) {
            const unsigned char* ys = yg(b);
            const unsigned char* ysn = yg(b + 1);
            const T* wst = reinterpret_cast<const T*>(wg(b));
            float* wp = wpl(b);
            float* upn = upl(b + 1);
            const unsigned ob = (unsigned)b * plane + o_t;
            w_item(Set0{}, ys, wst, wp, r_t, c_t, valid_t ? a.w1_n + ob : nullptr);
            w_item(Set1{}, ys, wst, wp, r_t, c_t, valid_t ? a.w2_n + ob : nullptr);
            if (has_next) u_item(ysn, upn, b + 1, r_t, c_t, (valid_t && b + 1 < b1) ? a.u_n + (ob + plane) : nullptr);
            if (has_rw) {
                if (rw_set == 0) w_item(Set0{}, ys, wst, wp, rw_r, rw_c, nullptr);
                else w_item(Set1{}, ys, wst, wp, rw_r, rw_c, nullptr);
            }
            if (has_ru && has_next) u_item(ysn, upn, b + 1, ru_r, ru_c, nullptr);
        }
        if (b > b0) t_item(b - 1);
        // the slots freed at this step are reloaded by TMA at the next one:
        // order this thread's generic accesses before those async-proxy writes
        fence_proxy_async_smem();
        if (__syncthreads_or(!okb)) return false;
    }
    t_item(b1 - 1);
    return true;
}

template <typename T>
__global__ void __launch_bounds__(512, 1) k1_tma(const __grid_constant__ K1Maps maps, const K1TArgs<T> a) {
    using L = Lay<T>;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ double red_d[64];
    __shared__ unsigned long long red_u[64];
    __shared__ int is_last;
    const Geom& g = a.g;
    const IterParams& P = a.p;
    const int i0 = blockIdx.y * L::TY, j0 = blockIdx.x * L::TX;
    const int b0 = blockIdx.z * a.chunk;
    const int b1 = min(g.n3, b0 + a.chunk);
    const int tid = threadIdx.x;
    const float cs = (float)(1.0 - a.sc->c[P.parity]);
    const bool win_s = !P.tau_exact && a.sc->radius[0] > 0.0 && a.sc->ctl[0].window_ok;
    const bool win_t = !P.tau_exact && a.sc->radius[1] > 0.0 && a.sc->ctl[1].window_ok;
    const float lo_s = a.sc->ctl[0].theta_lo, hi_s = a.sc->ctl[0].theta_hi;
    const float lo_t = a.sc->ctl[1].theta_lo, hi_t = a.sc->ctl[1].theta_hi;

    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L::OFF_BAR);
    if (tid == 0) {
        for (int k = 0; k < L::NYS + L::NWS; ++k) mbar_init(bars + k, 1);
        mbar_fence_init();
    }
    __syncthreads();

    K1State S;
    const bool edge = !(i0 >= 2 && i0 + L::TY + 3 <= g.n1 && j0 >= 2 && j0 + L::TX + 3 <= g.n2);
    bool ok = edge ? k1_tile<T, true>(maps, a, sm, i0, j0, b0, b1, S, win_s, win_t, lo_s, hi_s, lo_t, hi_t, cs)
                   : k1_tile<T, false>(maps, a, sm, i0, j0, b0, b1, S, win_s, win_t, lo_s, hi_s, lo_t, hi_t, cs);
    if (!ok) {
        // a load never arrived: record it, let this CTA's copies land (bounded)
        // before its shared memory is released, and skip the statistics
        if (tid == 0) {
            atomicOr(&a.sc->error, 4);
            for (int k = 0; k < L::NYS; ++k)
                if (S.n_y > (unsigned)k) (void)mbar_wait(bars + k, ((S.n_y - 1 - k) / L::NYS) & 1);
            for (int k = 0; k < L::NWS; ++k)
                if (S.n_w > (unsigned)k)
                    (void)mbar_wait(bars + L::NYS + k, ((S.n_w - 1 - k) / L::NWS) & 1);
        }
        __syncthreads();
    }

    const int cta = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int ncta = gridDim.x * gridDim.y * gridDim.z;
    if (win_s || win_t) {
        const unsigned long long ns = block_sum(S.acc_s.n, red_u);
        const double ss = block_sum(S.acc_s.s.value(), red_d);
        const unsigned long long nt = block_sum(S.acc_t.n, red_u);
        const double st = block_sum(S.acc_t.s.value(), red_d);
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
                C.tau = __int_as_float(0x7f800000);
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
        for (int k = tid; k < ncta; k += L::NT) {
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
                l1_record_tau(C, tau, (double)min(m, kCandCap), thi - tlo);
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

int tma_chunk(const Geom& g, int tiles) {
    int chunks = (152 * 12 + tiles - 1) / tiles;            // about 12 CTAs per SM over the launch
    chunks = std::max(1, std::min(chunks, (g.n3 + 7) / 8));
    return (g.n3 + chunks - 1) / chunks;
}

template <typename T>
int launch_k1_tma_t(const Geom& g, const K1Maps& m, const IterBufs& b, const IterParams& p, Scal* sc,
                    const L1Work& w, cudaStream_t st) {
    using L = Lay<T>;
    K1TArgs<T> a;
    a.g = g;
    a.u_n = (T*)b.u_n; a.w1_n = (T*)b.w1_n; a.w2_n = (T*)b.w2_n; a.y1_n = (T*)b.y1_n; a.y2_n = (T*)b.y2_n;
    a.p = p;
    a.sc = sc;
    a.l1 = w;
    const int tx = (g.n2 + L::TX - 1) / L::TX, ty = (g.n1 + L::TY - 1) / L::TY;
    a.chunk = tma_chunk(g, tx * ty);
    dim3 grid(tx, ty, (g.n3 + a.chunk - 1) / a.chunk);
    k1_tma<T><<<grid, L::NT, L::SMEM, st>>>(m, a);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace

int k1_tma_ctas(const Geom& g) {
    const int tx = (g.n2 + 31) / 32, ty = (g.n1 + 15) / 16;
    const int chunk = tma_chunk(g, tx * ty);
    return tx * ty * ((g.n3 + chunk - 1) / chunk);
}

// The TMA-fed kernel is built for float32 storage only (16-bit storage runs
// the cooperative-load kernel of k_stencil.cu).
int k1_tma_configure(int storage) {
    if (storage != 0) return -1;
    const cudaError_t e =
        cudaFuncSetAttribute(k1_tma<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, Lay<float>::SMEM);
    return e == cudaSuccess ? 0 : -3;
}

// tensor maps over the current-parity buffers of one iteration
int k1_tma_maps(int storage, const Geom& g, const IterBufs& b, K1Maps* m) {
    if (storage != 0) return -1;
    const int es = 4;
    const int ox = 16 / es, sw = 32 + 2 * ox;
    int rc = 0;
    rc |= tma_encode_cubes(&m->y1, b.y1, es, g.n1, g.n2, g.n3, g.p2, 2, sw, 16 + 4);
    rc |= tma_encode_cubes(&m->y2, b.y2, es, g.n1, g.n2, g.n3, g.p2, 2, sw, 16 + 4);
    rc |= tma_encode_cubes(&m->w1, b.w1, es, g.n1, g.n2, g.n3, g.p2, 6, sw, 16 + 2);
    rc |= tma_encode_cubes(&m->w2, b.w2, es, g.n1, g.n2, g.n3, g.p2, 6, sw, 16 + 2);
    rc |= tma_encode_cubes(&m->u, b.u, es, g.n1, g.n2, g.n3, g.p2, 1, sw, 16 + 1);
    rc |= tma_encode_cubes(&m->q, b.q, es, g.n1, g.n2, g.n3, g.p2, 1, sw, 16 + 1);
    rc |= tma_encode_cubes(&m->s, b.s, es, g.n1, g.n2, g.n3, g.p2, 1, 32, 16);
    rc |= tma_encode_cubes(&m->t, b.t, es, g.n1, g.n2, g.n3, g.p2, 1, 32, 16);
    rc |= tma_encode_cubes(&m->y3, b.y3, es, g.n1, g.n2, g.n3, g.p2, 1, 32, 16 + 1);
    return rc ? -3 : 0;
}

int launch_k1_tma(int storage, const Geom& g, const K1Maps& m, const IterBufs& b, const IterParams& p,
                  Scal* sc, const L1Work& w, cudaStream_t st) {
    return storage == 0 ? launch_k1_tma_t<float>(g, m, b, p, sc, w, st) : -1;
}

}  // namespace gsstv
