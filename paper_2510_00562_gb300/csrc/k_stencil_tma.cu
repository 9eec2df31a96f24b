// K1, TMA-fed: the fused stencil pass of one P-PDS iteration (Algorithm 1),
// float32 storage.
//
// Same arithmetic as the cooperative-load kernel in k_stencil.cu (u step and
// u' for band b+1; w1, w2 group soft-thresholds and w' on the tile plus a
// one-pixel ring; y1, y2 ascent; window statistics of the l1 threshold
// search), fed differently: each band's planes are brought into shared memory
// by bulk tensor (TMA) copies that one thread issues two bands ahead,
// completing on mbarriers.  One CTA of 512 threads per SM owns a 16 x 32 tile
// and a run of bands.  Tiles whose halo stays off the image border take a
// specialised path with no boundary masks.  Each CTA leaves its window
// statistics and candidates (with their key histogram) for the finishing
// launch that follows (k_search_finish, one CTA per vector), so that no CTA
// of this launch runs the threshold search while the rest of the GPU idles.
//
// Band march, one CTA barrier per band: while the w steps, u' of band b+1 and
// the window statistics of band b run, the dual ascent of band b-1 (which
// reads the w' and u' that the previous step completed) runs beside them.
// Each thread keeps the four y values of its own voxel that the ascent needs
// in registers for one band, so a y-group slot is free again as soon as its
// band's w step is done: 3 y-group slots (y1, y2 with a 2-pixel halo, u and q
// with a 1-pixel halo below/right, s, t, y3 with one row above) and 4 slots of
// the 12 w planes (1-pixel halo, w' written in place) fit beside u' of three
// bands and D^T y2 of the previous band: about 216 KB of shared memory.
#include <algorithm>
#include <vector>
#include <cmath>
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

constexpr int pad128(int b) { return (b + 127) / 128 * 128; }

struct Lay {
    static constexpr int TY = 16, TX = 32, NT = 512;
    static constexpr int OX = 4;                   // left halo columns: boxes start 16-byte aligned
    static constexpr int SW = TX + 2 * OX;         // width of the staged planes
    // the thread that issues the bulk copies: lane 0 of warp 8, a warp with no
    // ring items (the ring warps are 0-7, 10 and 15), so the serial copy issue
    // does not lengthen the slowest warp of a band step
    static constexpr int PRODUCER = 256;
    static constexpr int YR = TY + 4, WR = TY + 2, UR = TY + 1, UC = TX + 1;
    static constexpr int Y_B = pad128(YR * SW * 4);
    static constexpr int W_B = pad128(WR * SW * 4);
    static constexpr int U_B = pad128(UR * SW * 4);
    static constexpr int S_B = pad128(TY * TX * 4);
    static constexpr int Y3_B = pad128((TY + 1) * TX * 4);
    static constexpr int YG_B = 4 * Y_B + 2 * U_B + 2 * S_B + Y3_B;
    static constexpr int WG_B = 12 * W_B;
    static constexpr int NYS = 3, NWS = 4, NUS = 3;  // ring depths: y-group, w, u'
    static constexpr int UP1 = UR * UC;              // floats of one u' plane
    static constexpr int UP_B = pad128(NUS * UP1 * 4);
    static constexpr int G_B = pad128(UR * UC * 4);
    static constexpr int CB = 256;                   // window candidates buffered per CTA and vector
    static constexpr int OFF_WG = NYS * YG_B;
    static constexpr int OFF_UP = OFF_WG + NWS * WG_B;
    static constexpr int OFF_G = OFF_UP + UP_B;
    static constexpr int OFF_CB = OFF_G + G_B;
    static constexpr int OFF_HIST = OFF_CB + 2 * CB * 4;      // K1 histogram: 2 x kK1Bins packed 16-bit counts
    static constexpr int OFF_BAR = OFF_HIST + kK1Bins * 4;
    static constexpr int SMEM = OFF_BAR + (NYS + NWS) * 8;
    // float offsets inside a y-group slot, and between planes
    static constexpr int YPL = Y_B / 4, WPL = W_B / 4;
    static constexpr int O_U = 4 * YPL, O_Q = O_U + U_B / 4, O_S = O_Q + U_B / 4, O_T = O_S + S_B / 4,
                         O_Y3 = O_T + S_B / 4;
    // bytes each group's copies deliver
    static constexpr unsigned YG_TX = 4u * YR * SW * 4 + 2u * UR * SW * 4 + 2u * TY * TX * 4 + (TY + 1u) * TX * 4;
    static constexpr unsigned WG_TX = 12u * WR * SW * 4;
    // one-pixel ring: w positions 2 (TX + 2) + 2 TY per set, u' positions (TX + 1) + TY
    static constexpr int NWR = 2 * (TX + 2) + 2 * TY, NUR = (TX + 1) + TY;
    static_assert(TY * TX == NT, "one tile voxel per thread");
    // dynamic plus the kernel's static shared memory (the candidate counters:
    // 128 bytes, see ptxas -v) within the 227 KB a CTA may use
    static_assert(SMEM + 256 <= 227 * 1024, "shared memory");
    // the ring work layout (see k1_tile): per set 4 warps of 4 + 4 column and
    // 17 row items; the u' ring on 2 warps of 8 column items and at most 17
    // row items
    static_assert(NWR == 4 * (4 + 4 + 17) && TY == 16 && NUR == 2 * 8 + (TX + 1) && TX + 1 <= 2 * 17,
                  "ring work layout");
};

struct K1TArgs {
    Geom g;
    float *u_n, *w1_n, *w2_n, *y1_n, *y2_n;
    IterParams p;
    Scal* sc;
    L1Work l1;
    int chunk;
    SlabPart sp;
    int hist_fits;      // every CTA of the stage counts at most 65535 voxels
};

// Window of the l1 threshold search for this launch (see gsstv_l1.cuh), and
// the histograms of |s~|, |t~| near the predicted thresholds when they are on.
struct K1Win {
    bool s, t;
    float lo_s, hi_s, lo_t, hi_t;
    bool hs, ht;
    unsigned hb_s, hb_t;
    // the candidate lists' key histograms over the windows (null: not kept)
    unsigned *nh_s, *nh_t;
    NarrowGeom ng_s, ng_t;
};

// A thread's window statistics: count (a CTA covers at most a few thousand
// voxels per thread slot, so 32 bits suffice) and compensated sum.
struct K1Acc {
    unsigned n = 0;
    Kahan s;
};

// Per-CTA running state shared by the two tile paths.
struct K1State {
    K1Acc acc_s, acc_t;
    float2 ks = make_float2(0.f, 0.f), kc = make_float2(0.f, 0.f);   // packed window sums (s, t)
    K1Acc top_s, top_t;          // |x| above the histogram's range
    unsigned n_y = 0, n_w = 0;   // groups issued so far (thread 0 only)
};

// Appends the lanes' window candidates to the CTA's shared buffer (one
// shared-memory atomic per warp); values past its end go straight to the
// global list (and are not counted into its key histogram, so that the finish
// then bins the list itself: counting them here made K1 2 % slower).  `cnt`
// keeps counting past the buffer.
__device__ __forceinline__ void append_shared(bool take, float x, float* buf, unsigned* cnt, float* cand,
                                              unsigned* gcnt) {
    const unsigned mask = __ballot_sync(0xffffffffu, take);
    if (mask == 0) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(cnt, (unsigned)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    const unsigned k = base + __popc(mask & ((1u << lane) - 1u));
    if (take && k < (unsigned)Lay::CB) buf[k] = x;
    if (base + __popc(mask) > (unsigned)Lay::CB) {
        const bool over = take && k >= (unsigned)Lay::CB;
        append_candidate(over, x, cand, gcnt);
    }
}

// Counts x into the CTA's histogram (bins of the float key >> kHistShift from
// hb; two 16-bit counters per shared word), or into the above-range
// accumulator; values below the range are not needed.
__device__ __forceinline__ void hist_add(bool on, float x, unsigned hb, unsigned* h, K1Acc& top) {
    const unsigned kb = __float_as_uint(x) >> kHistShift;
    const unsigned bin = kb - hb;                    // below the range wraps to a large value
    const bool in = on && bin < (unsigned)kK1Bins;
    if (in) atomicAdd(h + (bin >> 1), (bin & 1u) ? 65536u : 1u);
    // above the range: an estimate from a sample, a plain sum suffices
    const bool up = on && !in && kb >= hb + (unsigned)kK1Bins;
    top.n += up ? 1u : 0u;
    top.s.s += up ? x : 0.f;
}

// value of a set selector: an int, or a std::integral_constant
template <typename X> __device__ __forceinline__ constexpr int set_of(X x) {
    if constexpr (std::is_integral<X>::value) return x;
    else return X::value;
}

// Packed FP32 pairs (two lanes per instruction on sm_100 and later), used for
// the (vertical, horizontal) pairs of the stencil; each lane rounds exactly as
// the scalar operation would.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f, -1.f), a); }

using Set0 = std::integral_constant<int, 0>;
using Set1 = std::integral_constant<int, 1>;
using Store = std::true_type;
using NoStore = std::false_type;

template <bool EDGE, bool HIST>
__device__ __forceinline__ bool k1_tile(const K1Maps& M, const K1TArgs& a, unsigned char* sm, unsigned* ccnt,
                                        int i0, int j0, int b0, int b1, K1State& S, const K1Win& W, float cs) {
    using L = Lay;
    constexpr int TY = L::TY, TX = L::TX, SW = L::SW, OX = L::OX, UC = L::UC;
    constexpr int YPL = L::YPL, WPL = L::WPL;
    const Geom& g = a.g;
    const IterParams& P = a.p;
    const int tid = threadIdx.x;
    const unsigned cube = (unsigned)g.cube;        // 6 cubes < 2^32 elements (checked at handle creation)
    const unsigned plane = (unsigned)g.n1 * (unsigned)g.p2;
    uint64_t* ybar = reinterpret_cast<uint64_t*>(sm + L::OFF_BAR);
    uint64_t* wbar = ybar + L::NYS;
    float* up = reinterpret_cast<float*>(sm + L::OFF_UP);
    float* gs = reinterpret_cast<float*>(sm + L::OFF_G);
    float* cbuf = reinterpret_cast<float*>(sm + L::OFF_CB);
    unsigned* hsm = reinterpret_cast<unsigned*>(sm + L::OFF_HIST);
    const int bstart = max(b0 - 1, 0);
    const int blast = min(b1, g.n3 - 1);

    // ---- ring slots ----
    auto ygb = [&](int band) { return sm + ((unsigned)(band - bstart) % L::NYS) * L::YG_B; };
    auto wgb = [&](int band) { return sm + L::OFF_WG + ((unsigned)(band - b0) % L::NWS) * L::WG_B; };
    auto yg = [&](int band) { return reinterpret_cast<const float*>(ygb(band)); };
    auto wg = [&](int band) { return reinterpret_cast<float*>(wgb(band)); };
    auto upl = [&](int band) { return up + ((unsigned)band % L::NUS) * L::UP1; };

    auto issue_y = [&](int band) {
        unsigned char* s = ygb(band);
        uint64_t* bar = ybar + (band - bstart) % L::NYS;
        mbar_arrive_expect_tx(bar, L::YG_TX);
        tma_load_3d(s + 0 * L::Y_B, &M.y1, j0 - OX, i0 - 2, band, bar);
        tma_load_3d(s + 1 * L::Y_B, &M.y1, j0 - OX, i0 - 2, g.n3 + band, bar);
        tma_load_3d(s + 2 * L::Y_B, &M.y2, j0 - OX, i0 - 2, band, bar);
        tma_load_3d(s + 3 * L::Y_B, &M.y2, j0 - OX, i0 - 2, g.n3 + band, bar);
        tma_load_3d(s + 4 * L::O_U, &M.u, j0 - OX, i0, band, bar);
        tma_load_3d(s + 4 * L::O_Q, &M.q, j0 - OX, i0, band, bar);
        tma_load_3d(s + 4 * L::O_S, &M.s, j0, i0, band, bar);
        tma_load_3d(s + 4 * L::O_T, &M.t, j0, i0, band, bar);
        tma_load_3d(s + 4 * L::O_Y3, &M.y3, j0, i0 - 1, band, bar);
        S.n_y++;
    };
    auto issue_w = [&](int band) {
        unsigned char* s = wgb(band);
        uint64_t* bar = wbar + (band - b0) % L::NWS;
        mbar_arrive_expect_tx(bar, L::WG_TX);
        for (int k = 0; k < 6; ++k) tma_load_3d(s + k * L::W_B, &M.w1, j0 - OX, i0 - 1, k * g.n3 + band, bar);
        for (int k = 0; k < 6; ++k) tma_load_3d(s + (6 + k) * L::W_B, &M.w2, j0 - OX, i0 - 1, k * g.n3 + band, bar);
        S.n_w++;
    };
    auto wait_y = [&](int band) {
        return mbar_wait(ybar + (unsigned)(band - bstart) % L::NYS, ((unsigned)(band - bstart) / L::NYS) & 1);
    };
    auto wait_w = [&](int band) { return mbar_wait(wbar + (unsigned)(band - b0) % L::NWS, ((unsigned)(band - b0) / L::NWS) & 1); };

    // D^T y = D_v^T y_v + D_h^T y_h at tile-relative (r, c); yv, yh: y planes
    auto dty = [&](const float* yv, const float* yh, int r, int c) {
        const int k = (r + 2) * SW + (c + OX);
        if constexpr (EDGE) {
            const int gi = i0 + r, gj = j0 + c;
            float d = 0.f;
            if (gi >= 1) d += yv[k - SW];
            if (gi <= g.n1 - 2) d -= yv[k];
            if (gj >= 1) d += yh[k - 1];
            if (gj <= g.n2 - 2) d -= yh[k];
            return d;
        } else {
            return ((yv[k - SW] - yv[k]) + yh[k - 1]) - yh[k];
        }
    };
    // u step and u' of band bb at (r, c) in [0, TY] x [0, TX]; ys: y-group of
    // bb; upb: u' plane of bb; with Store, u+ goes to *dst when `st`
    auto u_item = [&](auto store_c, const float* ys, float* upb, int bb, int r, int c, float* dst, bool st) {
        const int kc = r * UC + c;
        if constexpr (EDGE) {
            if (i0 + r >= g.n1 || j0 + c >= g.n2) { upb[kc] = 0.f; gs[kc] = 0.f; return; }
        }
        float d1, gcur;                                 // D^T y1 and D^T y2 of the band
        if constexpr (EDGE) {
            d1 = dty(ys, ys + YPL, r, c);
            gcur = dty(ys + 2 * YPL, ys + 3 * YPL, r, c);
        } else {
            const int k = (r + 2) * SW + (c + OX);
            const float *v1 = ys + k, *h1 = ys + YPL + k, *v2 = ys + 2 * YPL + k, *h2 = ys + 3 * YPL + k;
            const float2 d = sub2(add2(sub2(f2(v1[-SW], v2[-SW]), f2(v1[0], v2[0])), f2(h1[-1], h2[-1])), f2(h1[0], h2[0]));
            d1 = d.x;
            gcur = d.y;
        }
        // D_s^T at the band's place in the whole cube (Neumann at its ends)
        const float gprev = gs[kc];
        const int gb = bb + a.sp.band0;
        float dst_ = 0.f;
        if (gb >= 1) dst_ += gprev;
        if (gb <= a.sp.n3g - 2) dst_ -= gcur;
        const int ku = r * SW + (c + OX);
        const float y4 = cs * ys[L::O_Q + ku];
        const float u = ys[L::O_U + ku];
        const float un = fminf(fmaxf(u - P.gamma_u * (d1 + dst_ + y4), P.mu_lo), P.mu_hi);
        upb[kc] = 2.f * un - u;
        gs[kc] = gcur;
        if constexpr (decltype(store_c)::value) {
            if (st) *dst = un;
        }
    };
    // w step of one set (0 = w1, 1 = w2; a compile-time constant or not) at
    // (r, c) in [-1, TY] x [-1, TX]; w' overwrites w in place; with Store, w+
    // goes to dst (the set's first plane) when `st`
    auto w_item = [&](auto set_c, auto store_c, const float* ys, float* wst, int r, int c, float* dst, bool st) {
        const int set = set_of(set_c);
        const int kw = (r + 1) * SW + (c + OX);
        const int gi = i0 + r, gj = j0 + c;
        if constexpr (EDGE) {
            if (gi < 0 || gi >= g.n1 || gj < 0 || gj >= g.n2) {
#pragma unroll
                for (int k = 0; k < 6; ++k) wst[(6 * set + k) * WPL + kw] = 0.f;
                return;
            }
        }
        const bool mv = !EDGE || gi < g.n1 - 1, mh = !EDGE || gj < g.n2 - 1;
        const int ky = (r + 2) * SW + (c + OX);
        const float* yv = ys + (2 * set) * YPL + ky;
        const float* yh = yv + YPL;
        auto V = [&](int dr, int dc) {
            if constexpr (EDGE) return (gi + dr == g.n1 - 1) ? 0.f : yv[dr * SW + dc];
            else return yv[dr * SW + dc];
        };
        auto H = [&](int dr, int dc) {
            if constexpr (EDGE) return (gj + dc == g.n2 - 1) ? 0.f : yh[dr * SW + dc];
            else return yh[dr * SW + dc];
        };
        const float v00 = V(0, 0), vm0 = V(-1, 0), v01 = V(0, 1), vm1 = V(-1, 1);
        const float h00 = H(0, 0), h0m = H(0, -1), h10 = H(1, 0), h1m = H(1, -1);
        // (v, h) pairs: the centred means 0.5 (v00 + vm0), 0.5 (h00 + h0m), and
        // the four-point means 0.25 (v00 + vm0 + v01 + vm1), 0.25 (h00 + h0m + h10 + h1m)
        float2 sum = add2(f2(v00, h00), f2(vm0, h0m));
        const float2 cen = mul2(sum, f2(0.5f, 0.5f));
        sum = add2(add2(sum, f2(v01, h10)), f2(vm1, h1m));
        const float2 four = mul2(sum, f2(0.25f, 0.25f));
        float2 Lg[3];                                   // (L_v, L_h) of the three grids
        Lg[0] = f2(mv ? v00 : 0.f, mv ? four.y : 0.f);
        Lg[1] = f2(mh ? four.x : 0.f, mh ? h00 : 0.f);
        Lg[2] = cen;
        const float gam = set ? P.gamma_w2 : P.gamma_w1;
        const float thr = set ? P.thr_w2 : P.thr_w1;
        const float thr2 = thr * thr;
        float* wp = wst + (6 * set) * WPL + kw;
#pragma unroll
        for (int gr = 0; gr < 3; ++gr) {
            const float wv = wp[(2 * gr) * WPL];
            const float wh = wp[(2 * gr + 1) * WPL];
            const float2 x = fma2(f2(gam, gam), Lg[gr], f2(wv, wh));
            const float xv = x.x, xh = x.y;
            // Eq. 24: max(1 - thr / ||x||, 0) x, with 1 / ||x|| from rsqrt
            const float n2 = xv * xv + xh * xh;
            const float sc = n2 > thr2 ? fmaxf(1.f - thr * rsqrtf(n2), 0.f) : 0.f;
            const float2 nn = mul2(f2(sc, sc), x);
            const float nv = nn.x, nh = nn.y;
            wp[(2 * gr) * WPL] = 2.f * nv - wv;
            wp[(2 * gr + 1) * WPL] = 2.f * nh - wh;
            if constexpr (decltype(store_c)::value) {
                if (st) {
                    dst[(2 * gr) * cube] = nv;
                    dst[(2 * gr + 1) * cube] = nh;
                }
            }
        }
    };

    // ---- this thread's tile voxel and its share of the one-pixel ring ----
    const int r_t = tid / TX, c_t = tid - (tid / TX) * TX;
    const int gi_t = i0 + r_t, gj_t = j0 + c_t;
    const bool valid_t = !EDGE || (gi_t < g.n1 && gj_t < g.n2);
    const unsigned o_t = valid_t ? (unsigned)gi_t * (unsigned)g.p2 + (unsigned)gj_t : 0u;
    const int ky_t = (r_t + 2) * SW + (c_t + OX);
    // The one-pixel ring: w items on warps 0-7, u' items on warps 10 and 15
    // (each scheduler, warp index mod 4, gets two or three ring warps besides
    // its four tile warps).  A column of the ring walks rows 40 floats apart,
    // so rows r and r + 4 fall in one shared-memory bank: a w warp takes four
    // consecutive rows of each column, a u' warp eight (the mapping that gave
    // a warp all 16 rows of a column made K1 0.6 % slower through bank
    // conflicts).
    int rw_r = 0, rw_c = 0, ru_r = 0, ru_c = 0;
    const int wid = tid >> 5, lane = tid & 31;
    // w ring: warps 0-7, warp w holds set w / 4 and quarter q = w % 4 of it:
    // the left and right column items of rows 4q..4q+3 (distinct banks) and
    // 17 of the 68 row items
    const bool has_rw = wid < 8 && lane < 25;
    const int rw_set = wid >= 4 ? 1 : 0;
    if (has_rw) {
        const int q = wid & 3;
        if (lane < 4) { rw_r = 4 * q + lane; rw_c = -1; }
        else if (lane < 8) { rw_r = 4 * q + lane - 4; rw_c = TX; }
        else {
            const int ri = 17 * q + lane - 8;           // 0..67
            if (ri < TX + 2) { rw_r = -1; rw_c = ri - 1; } else { rw_r = TY; rw_c = ri - (TX + 2) - 1; }
        }
    }
    // u' ring: warps 10 and 15, each 8 right-column items and half the row
    const int uq = wid == 10 ? 0 : wid == 15 ? 1 : -1;
    const bool has_ru = uq >= 0 && lane < (uq == 0 ? 25 : 24);
    if (has_ru) {
        if (lane < 8) { ru_r = 8 * uq + lane; ru_c = TX; }
        else { ru_r = TY; ru_c = 17 * uq + lane - 8; }
    }

    // ---- dual ascent of y1, y2 at this thread's voxel of band tb ----
    // Reads the band's completed w' and u' of the band and the next; yc: the
    // voxel's y1 (v, h), y2 (v, h) of band tb.
    auto t_item = [&](int tb, const float (&yc)[4]) {
        if (!valid_t) return;
        const bool nxt = tb + 1 < g.n3;
        const float* upb = upl(tb);
        const float* upn = upl(tb + 1);
        const float* wp = wg(tb);
        const int kc = r_t * UC + c_t;
        const float u0 = upb[kc];
        const bool mv = !EDGE || gi_t < g.n1 - 1, mh = !EDGE || gj_t < g.n2 - 1;
        // (vertical, horizontal) pairs: D u' and D D_s u' at the voxel
        const float2 ub = f2(upb[kc + UC], upb[kc + 1]);
        const float2 du_ = sub2(ub, f2(u0, u0));
        const float2 du = f2(mv ? du_.x : 0.f, mh ? du_.y : 0.f);
        const float d0 = upn[kc] - u0;
        const float2 dd_ = sub2(sub2(f2(upn[kc + UC], upn[kc + 1]), ub), f2(d0, d0));
        const float2 dd = f2(nxt && mv ? dd_.x : 0.f, nxt && mh ? dd_.y : 0.f);
        const float* wk = wp + (r_t + 1) * SW + (c_t + OX);
        float2 lt[2];                                    // (L^T w')_v, (L^T w')_h of each set
#pragma unroll
        for (int set = 0; set < 2; ++set) {
            auto Wk = [&](int k, int dr, int dc) { return wk[(6 * set + k) * WPL + dr * SW + dc]; };
            auto A_ = [&](int dr, int dc) {
                if constexpr (EDGE) return (gi_t + dr < g.n1 - 1) ? Wk(1, dr, dc) : 0.f;
                else return Wk(1, dr, dc);
            };
            auto B_ = [&](int dr, int dc) {
                if constexpr (EDGE) return (gj_t + dc < g.n2 - 1) ? Wk(2, dr, dc) : 0.f;
                else return Wk(2, dr, dc);
            };
            // v: W0 + 0.25 (B(0,0) + B(1,0) + B(0,-1) + B(1,-1)) + 0.5 (W4(0,0) + W4(1,0))
            // h: W3 + 0.25 (A(0,0) + A(0,1) + A(-1,0) + A(-1,1)) + 0.5 (W5(0,0) + W5(0,1))
            const float2 s4 = add2(add2(add2(f2(B_(0, 0), A_(0, 0)), f2(B_(1, 0), A_(0, 1))), f2(B_(0, -1), A_(-1, 0))),
                                   f2(B_(1, -1), A_(-1, 1)));
            const float2 s2 = add2(f2(Wk(4, 0, 0), Wk(5, 0, 0)), f2(Wk(4, 1, 0), Wk(5, 0, 1)));
            const float2 gg = fma2(f2(0.5f, 0.5f), s2, fma2(f2(0.25f, 0.25f), s4, f2(Wk(0, 0, 0), Wk(3, 0, 0))));
            lt[set] = f2(mv ? gg.x : 0.f, mh ? gg.y : 0.f);
        }
        const unsigned ob = (unsigned)tb * plane + o_t;
        const float2 y1 = fma2(f2(P.gamma_y1, P.gamma_y1), sub2(du, lt[0]), f2(yc[0], yc[1]));
        const float2 y2 = fma2(f2(P.gamma_y2, P.gamma_y2), sub2(dd, lt[1]), f2(yc[2], yc[3]));
        a.y1_n[ob] = y1.x;
        a.y1_n[cube + ob] = y1.y;
        a.y2_n[ob] = y2.x;
        a.y2_n[cube + ob] = y2.y;
    };

    // ---- l1 window statistics of s~, t~ at this thread's voxel ----
    auto stats = [&](const float* ys, int b) {
        float xs = 0.f, xt = 0.f;
        if (valid_t) {
            // s~ = s - g_s y4, t~ = t - g_t (D_v^T y3 + y4), each product and
            // difference rounded once as in s_t_tilde (the light pass computes
            // the same values), the (s, t) pair packed
            const float qv = ys[L::O_Q + r_t * SW + (c_t + OX)];
            const float y3v = ys[L::O_Y3 + (r_t + 1) * TX + c_t];
            const float y3u = (!EDGE || gi_t >= 1) ? ys[L::O_Y3 + r_t * TX + c_t] : 0.f;
            const float y4 = __fmul_rn(cs, qv);
            const float dvt = __fsub_rn(y3u, gi_t <= g.n1 - 2 ? y3v : 0.f);
            const float2 m = mul2(f2(P.gamma_s, P.gamma_t), f2(y4, __fadd_rn(dvt, y4)));
            const float2 x = sub2(f2(ys[L::O_S + r_t * TX + c_t], ys[L::O_T + r_t * TX + c_t]), m);
            xs = x.x;
            xt = x.y;
        }
        // an inactive window has lo = hi = +inf: nothing is counted or taken
        const float x_s = fabsf(xs), x_t = fabsf(xt);
        const bool hs = valid_t && x_s > W.hi_s, ht = valid_t && x_t > W.hi_t;
        {
            // both vectors' compensated sums in packed pairs; a value not
            // taken adds zero, which leaves the represented sum unchanged
            const float2 x2 = f2(hs ? x_s : 0.f, ht ? x_t : 0.f);
            const float2 y2 = sub2(x2, S.kc);
            const float2 t2 = add2(S.ks, y2);
            S.kc = sub2(sub2(t2, S.ks), y2);
            S.ks = t2;
            S.acc_s.n += hs ? 1u : 0u;
            S.acc_t.n += ht ? 1u : 0u;
        }
        const bool cs_ = valid_t && !hs && x_s > W.lo_s, ct_ = valid_t && !ht && x_t > W.lo_t;
        if (__ballot_sync(0xffffffffu, cs_ || ct_)) {     // most warps have no candidate
            append_shared(cs_, x_s, cbuf, ccnt, a.l1.cand[0], &a.sc->acc[0].m);
            append_shared(ct_, x_t, cbuf + L::CB, ccnt + 1, a.l1.cand[1], &a.sc->acc[1].m);
        }
        if constexpr (HIST) {
            // a 1/32 sample: a warp (one row of the tile) counts its 32 voxels
            // at one band in 32, the band rotating with the row and the tile
            // so that every band is sampled; the branch is warp-uniform, so
            // the other 31 band steps cost one test
            if ((((unsigned)b + 7u * (unsigned)r_t + 5u * (unsigned)(i0 >> 4) + 3u * (unsigned)(j0 >> 5)) & 31u) == 0u) {
                hist_add(W.hs && valid_t, x_s, W.hb_s, hsm, S.top_s);
                hist_add(W.ht && valid_t, x_t, W.hb_t, hsm + kK1Bins / 2, S.top_t);
            }
        }
    };

    // ---- prologue: D^T y2 of band b0-1 and u' of band b0 ----
    if (tid == L::PRODUCER) {
        for (int band = bstart; band <= min(bstart + L::NYS - 1, blast); ++band) issue_y(band);
        issue_w(b0);
        if (b0 + 1 < b1) issue_w(b0 + 1);
    }
    bool ok = true;
    if (b0 >= 1) {
        ok = wait_y(b0 - 1);
        const float* yp = yg(b0 - 1);
        for (int e = tid; e < L::UR * UC; e += L::NT) {
            const int r = e / UC, c = e - r * UC;
            if (EDGE && (i0 + r >= g.n1 || j0 + c >= g.n2)) { gs[e] = 0.f; continue; }
            gs[e] = dty(yp + 2 * YPL, yp + 3 * YPL, r, c);
        }
    }
    ok = wait_y(b0) && ok;
    ok = __syncthreads_and(ok);
    if (!ok) return false;
    u_item(Store{}, yg(b0), upl(b0), b0, r_t, c_t, a.u_n + ((unsigned)b0 * plane + o_t), valid_t);
    if (has_ru) u_item(NoStore{}, yg(b0), upl(b0), b0, ru_r, ru_c, nullptr, false);
    __syncthreads();

    // ---- band march, one barrier per band ----
    // The ascent of the previous band needs nothing from this band's copies,
    // so it runs before the waits on them; then the tile work of the band
    // (the statistics, w steps, u' of the next band) is one straight run so
    // that the compiler can interleave its independent chains, and the ring
    // work follows.  u' of the band past the cube's last one is computed from
    // a stale slot and not stored (its values are never used).
    float yprev[4] = {0.f, 0.f, 0.f, 0.f};
    auto step = [&](int b, auto do_t) -> bool {
        const bool has_next = b + 1 < g.n3;
        if (tid == L::PRODUCER) {
            if (b + 2 <= blast && b + 2 - bstart >= L::NYS) issue_y(b + 2);
            if (b + 2 < b1) issue_w(b + 2);
        }
        if constexpr (decltype(do_t)::value) t_item(b - 1, yprev);
        bool okb = wait_w(b);
        if (has_next) okb = wait_y(b + 1) && okb;
        okb = __all_sync(0xffffffffu, okb);   // warp-uniform: the statistics use warp votes
        if (okb) {
            const float* ys = yg(b);
            const float* ysn = yg(b + 1);
            float* wst = wg(b);
            float* upn = upl(b + 1);
            const unsigned ob = (unsigned)b * plane + o_t;
            float ycur[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) ycur[k] = ys[k * YPL + ky_t];
            if (W.s || W.t) stats(ys, b);
            w_item(Set0{}, Store{}, ys, wst, r_t, c_t, a.w1_n + ob, valid_t);
            w_item(Set1{}, Store{}, ys, wst, r_t, c_t, a.w2_n + ob, valid_t);
            u_item(Store{}, ysn, upn, b + 1, r_t, c_t, a.u_n + (ob + plane), valid_t && b + 1 < b1);
            if (has_rw) w_item(rw_set, NoStore{}, ys, wst, rw_r, rw_c, nullptr, false);
            if (has_ru && has_next) u_item(NoStore{}, ysn, upn, b + 1, ru_r, ru_c, nullptr, false);
#pragma unroll
            for (int k = 0; k < 4; ++k) yprev[k] = ycur[k];
        }
        // the slots freed at this step are reloaded by TMA at the next one:
        // order this thread's generic accesses before those async-proxy writes
        fence_proxy_async_smem();
        return !__syncthreads_or(!okb);
    };
    if (!step(b0, std::false_type{})) return false;
    for (int b = b0 + 1; b < b1; ++b)
        if (!step(b, std::true_type{})) return false;
    t_item(b1 - 1, yprev);
    return true;
}

// One CTA of K1: the tile (bx, by) and band run bz of a launch of gx x gy x gz
// CTAs over one cube (a launch of its own, or the cube's share of a batch).
__device__ __forceinline__ void k1_run(const K1Maps& maps, const K1TArgs& a, const int bx, const int by,
                                       const int bz, const int gx, const int gy, const int gz) {
    using L = Lay;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ unsigned ccnt[2], cbase[2];
    const Geom& g = a.g;
    const IterParams& P = a.p;
    const int i0 = by * L::TY, j0 = bx * L::TX;
    const int b0 = a.sp.o0 + bz * a.chunk;
    const int b1 = min(a.sp.o1, b0 + a.chunk);
    const int tid = threadIdx.x;
    const float cs = (float)(1.0 - a.sc->c[P.parity]);
    K1Win W;
    W.s = !P.tau_exact && a.sc->radius[0] > 0.0 && a.sc->ctl[0].window_ok;
    W.t = !P.tau_exact && a.sc->radius[1] > 0.0 && a.sc->ctl[1].window_ok;
    W.lo_s = W.s ? a.sc->ctl[0].theta_lo : INFINITY; W.hi_s = W.s ? a.sc->ctl[0].theta_hi : INFINITY;
    W.lo_t = W.t ? a.sc->ctl[1].theta_lo : INFINITY; W.hi_t = W.t ? a.sc->ctl[1].theta_hi : INFINITY;
    // the histograms: on after a recent miss, while a CTA's voxels fit the
    // 16-bit counters
    const bool hist_fits = a.hist_fits != 0;
    W.hb_s = a.sc->ctl[0].hbase;
    W.hb_t = a.sc->ctl[1].hbase;
    W.hs = W.s && hist_fits && a.sc->ctl[0].hist_left > 0 && hist_base_ok(W.hb_s);
    W.ht = W.t && hist_fits && a.sc->ctl[1].hist_left > 0 && hist_base_ok(W.hb_t);
    W.ng_s = narrow_geom(__float_as_uint(W.lo_s), __float_as_uint(W.hi_s));
    W.ng_t = narrow_geom(__float_as_uint(W.lo_t), __float_as_uint(W.hi_t));
    W.nh_s = W.s && a.l1.nh && W.ng_s.ok ? a.l1.nh : nullptr;
    W.nh_t = W.t && a.l1.nh && W.ng_t.ok ? a.l1.nh + 3 * kNarrowBins : nullptr;

    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L::OFF_BAR);
    if (tid == 0) {
        for (int k = 0; k < L::NYS + L::NWS; ++k) mbar_init(bars + k, 1);
        mbar_fence_init();
        ccnt[0] = ccnt[1] = 0;
    }
    if (W.hs || W.ht) {
        unsigned* hsm = reinterpret_cast<unsigned*>(sm + L::OFF_HIST);
        for (int k = tid; k < kK1Bins; k += L::NT) hsm[k] = 0u;
    }
    __syncthreads();

    K1State S;
    const bool edge = !(i0 >= 2 && i0 + L::TY + 3 <= g.n1 && j0 >= 2 && j0 + L::TX + 3 <= g.n2);
    const bool hist = W.hs || W.ht;
    const bool ok = edge ? (hist ? k1_tile<true, true>(maps, a, sm, ccnt, i0, j0, b0, b1, S, W, cs)
                                 : k1_tile<true, false>(maps, a, sm, ccnt, i0, j0, b0, b1, S, W, cs))
                         : (hist ? k1_tile<false, true>(maps, a, sm, ccnt, i0, j0, b0, b1, S, W, cs)
                                 : k1_tile<false, false>(maps, a, sm, ccnt, i0, j0, b0, b1, S, W, cs));
    if (!ok) {
        // a load never arrived: record it, let this CTA's copies land (bounded)
        // before its shared memory is released, and skip the statistics (the
        // producer holds the counts of the copies it issued)
        if (tid == L::PRODUCER) {
            atomicOr(&a.sc->error, 4);
            for (int k = 0; k < L::NYS; ++k)
                if (S.n_y > (unsigned)k) (void)mbar_wait(bars + k, ((S.n_y - 1 - k) / L::NYS) & 1);
            for (int k = 0; k < L::NWS; ++k)
                if (S.n_w > (unsigned)k)
                    (void)mbar_wait(bars + L::NYS + k, ((S.n_w - 1 - k) / L::NWS) & 1);
        }
        __syncthreads();
    }

    // this CTA among every CTA of the pass stage (all slabs of a split cube)
    const int cta = a.sp.cta_base + bx + gx * (by + gy * bz);
    if (W.s || W.t) {
        // the buffered window candidates join the global list (one atomic per vector)
        __syncthreads();
        if (tid < 2) {
            const unsigned n = min(ccnt[tid], (unsigned)L::CB);
            cbase[tid] = n ? atomicAdd(&a.sc->acc[tid].m, n) : 0u;
        }
        __syncthreads();
        const float* cbuf = reinterpret_cast<const float*>(sm + L::OFF_CB);
        for (int v = 0; v < 2; ++v) {
            const unsigned n = min(ccnt[v], (unsigned)L::CB);
            for (unsigned k = tid; k < n; k += L::NT)
                if (cbase[v] + k < kCandCap) a.l1.cand[v][cbase[v] + k] = cbuf[v * L::CB + k];
            // and into the list's key histogram over the window, which the
            // finish then narrows without another pass over the candidates
            unsigned* h = v == 0 ? W.nh_s : W.nh_t;
            if (h) {
                const NarrowGeom& ng = v == 0 ? W.ng_s : W.ng_t;
                for (unsigned k = tid; k < n; k += L::NT) narrow_add(h, ng, __float_as_uint(cbuf[v * L::CB + k]));
                if (tid == 0 && n) atomicAdd(a.l1.nbinned + v, n);
            }
        }
        if (W.hs || W.ht) {
            // the histogram joins the global one (unpacked, nonzero bins only)
            const unsigned* hsm = reinterpret_cast<const unsigned*>(sm + L::OFF_HIST);
            for (int k = tid; k < kK1Bins; k += L::NT) {
                const unsigned w = hsm[k];
                const int v = k / (kK1Bins / 2), b = 2 * (k - v * (kK1Bins / 2));
                unsigned* gh = a.l1.khist + v * kK1Bins + b;
                if (w & 0xffffu) atomicAdd(gh, w & 0xffffu);
                if (w >> 16) atomicAdd(gh + 1, w >> 16);
            }
        }
        // the CTA's window statistics (counts and sums above the windows) and
        // the histograms' above-range statistics, reduced together: 32-bit
        // counts and float-pair sums through the warps, one barrier, thread 0
        // finishes (no FP64 outside thread 0)
        unsigned n4[4] = {S.acc_s.n, S.acc_t.n, S.top_s.n, S.top_t.n};
        float hi4[4] = {S.ks.x, S.ks.y, S.top_s.s.s, S.top_t.s.s};
        float lo4[4] = {-S.kc.x, -S.kc.y, -S.top_s.s.c, -S.top_t.s.c};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                n4[q] += __shfl_xor_sync(0xffffffffu, n4[q], o);
                const float bh = __shfl_xor_sync(0xffffffffu, hi4[q], o), bl = __shfl_xor_sync(0xffffffffu, lo4[q], o);
                pair_add(hi4[q], lo4[q], bh, bl);
            }
        }
        float* wbuf = reinterpret_cast<float*>(sm + L::OFF_G);          // idle now: 16 warps x 12 values
        if ((tid & 31) == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                wbuf[(tid >> 5) * 12 + q] = __uint_as_float(n4[q]);
                wbuf[(tid >> 5) * 12 + 4 + q] = hi4[q];
                wbuf[(tid >> 5) * 12 + 8 + q] = lo4[q];
            }
        }
        __syncthreads();
        if (tid == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                unsigned long long n = 0;
                float h = wbuf[4 + q], l = wbuf[8 + q];
                n += __float_as_uint(wbuf[q]);
                for (int w = 1; w < L::NT / 32; ++w) {
                    n += __float_as_uint(wbuf[w * 12 + q]);
                    pair_add(h, l, wbuf[w * 12 + 4 + q], wbuf[w * 12 + 8 + q]);
                }
                a.l1.k1_n[4 * cta + q] = n;
                a.l1.k1_s[4 * cta + q] = (double)h + (double)l;
            }
        }
    }
    // what this pass counted, for the finishing launch that follows (every
    // CTA agrees; the first writes it)
    if (cta == 0 && tid == 0) {
        a.sc->k1_win[0] = W.s; a.sc->k1_win[1] = W.t;
        a.sc->k1_hist[0] = W.hs; a.sc->k1_hist[1] = W.ht;
    }
}

__global__ void __launch_bounds__(512, 1) k1_tma(const __grid_constant__ K1Maps maps, const K1TArgs a) {
    k1_run(maps, a, blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x, gridDim.y, gridDim.z);
}

// K1 over many cubes in one launch: the cube of a CTA from a table of first
// CTAs, its arguments from the table, its tensor maps from device memory.
struct K1BatchTab {
    int n;
    int start[kBatchMax + 1];
    short gx[kBatchMax], gy[kBatchMax], gz[kBatchMax];
    const K1Maps* maps[kBatchMax];
    K1TArgs args[kBatchMax];
};

__device__ __forceinline__ int batch_cube_of(const int* start, int n, int blk) {
    int lo = 0, hi = n - 1;                 // the last cube whose first CTA is <= blk
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= blk) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(512, 1) k1_tma_batch(const __grid_constant__ K1BatchTab t) {
    const int c = batch_cube_of(t.start, t.n, blockIdx.x);
    // the cube's arguments by value: the table is indexed by a run-time
    // cube, so each field is loaded once instead of at each use
    const K1TArgs a = t.args[c];
    if (__ldcg(&a.sc->done)) return;        // this cube has stopped
    const int gx = t.gx[c], gy = t.gy[c], gz = t.gz[c];
    const int l = blockIdx.x - t.start[c];
    const int bx = l % gx, by = (l / gx) % gy, bz = l / (gx * gy);
    const K1Maps* maps = t.maps[c];
    if (threadIdx.x == Lay::PRODUCER) {
        // the cube's tensor maps sit in global memory (the copies' descriptors)
        tma_prefetch_map(&maps->y1); tma_prefetch_map(&maps->y2); tma_prefetch_map(&maps->w1);
        tma_prefetch_map(&maps->w2); tma_prefetch_map(&maps->u); tma_prefetch_map(&maps->q);
        tma_prefetch_map(&maps->s); tma_prefetch_map(&maps->t); tma_prefetch_map(&maps->y3);
    }
    k1_run(*maps, a, bx, by, bz, gx, gy, gz);
}

// Bands per CTA.  One CTA runs per SM, so a launch of U CTAs on S SMs takes
// ceil(U / S) waves and the last wave leaves SMs idle; every CTA also pays a
// prologue of about 1.5 band steps (its first copies, D^T y2 of the band
// before, u' of its first band).  Picks the split of the bands (runs of at
// least 8) that minimises idle fraction + prologue fraction.
int tma_chunk(int nb, int tiles) {
    const double kSms = (double)device_sms();
    constexpr double kPrologue = 1.5;
    const int max_chunks = std::max(1, nb / 8);
    int best_len = nb;
    double best = 1e30;
    for (int chunks = 1; chunks <= max_chunks; ++chunks) {
        const int len = (nb + chunks - 1) / chunks;
        const int used = (nb + len - 1) / len;                 // chunks actually launched
        const double units = (double)tiles * used;
        const double waves = std::ceil(units / kSms);
        const double waste = (waves - units / kSms) / waves + kPrologue / len;
        if (waste < best - 1e-12) { best = waste; best_len = len; }
    }
    return best_len;
}

}  // namespace

// CTAs of the largest launch any allowed band run gives (runs of at least 8
// bands, or all of them when there are fewer): the per-CTA statistics arrays
// are sized for it.
int k1_tma_ctas(const Geom& g) {
    const int tx = (g.n2 + Lay::TX - 1) / Lay::TX, ty = (g.n1 + Lay::TY - 1) / Lay::TY;
    const int shortest = std::min(8, g.n3);
    return tx * ty * ((g.n3 + shortest - 1) / shortest);
}

// Run lengths worth timing: the model's choice and the next best by its
// estimate, at most `cap` distinct lengths, the model's choice first.
int k1_tma_chunk_candidates(const Geom& g, int* out, int cap) {
    const double kSms = (double)device_sms();
    constexpr double kPrologue = 1.5;
    const int tx = (g.n2 + Lay::TX - 1) / Lay::TX, ty = (g.n1 + Lay::TY - 1) / Lay::TY;
    const int tiles = tx * ty;
    const int max_chunks = std::max(1, g.n3 / 8);
    std::vector<std::pair<double, int>> c;
    for (int chunks = 1; chunks <= max_chunks; ++chunks) {
        const int len = (g.n3 + chunks - 1) / chunks;
        if (!c.empty() && c.back().second == len) continue;
        const int used = (g.n3 + len - 1) / len;
        const double units = (double)tiles * used;
        const double waves = std::ceil(units / kSms);
        c.push_back({(waves - units / kSms) / waves + kPrologue / len, len});
    }
    std::stable_sort(c.begin(), c.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
    const int first = tma_chunk(g.n3, tiles);
    int n = 0;
    if (cap > 0) out[n++] = first;
    for (const auto& e : c)
        if (n < cap && e.second != first) out[n++] = e.second;
    return n;
}

// The TMA-fed kernel is built for float32 storage only (16-bit storage runs
// the cooperative-load kernel of k_stencil.cu).
int k1_tma_configure(int storage) {
    if (storage != 0) return -1;
    const cudaError_t e = cudaFuncSetAttribute(k1_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, Lay::SMEM);
    return e == cudaSuccess ? 0 : -3;
}

// tensor maps over the current-parity buffers of one iteration
int k1_tma_maps(int storage, const Geom& g, const IterBufs& b, K1Maps* m) {
    if (storage != 0) return -1;
    constexpr int sw = Lay::SW, ty = Lay::TY;
    int rc = 0;
    rc |= tma_encode_cubes(&m->y1, b.y1, 4, g.n1, g.n2, g.n3, g.p2, 2, sw, ty + 4);
    rc |= tma_encode_cubes(&m->y2, b.y2, 4, g.n1, g.n2, g.n3, g.p2, 2, sw, ty + 4);
    rc |= tma_encode_cubes(&m->w1, b.w1, 4, g.n1, g.n2, g.n3, g.p2, 6, sw, ty + 2);
    rc |= tma_encode_cubes(&m->w2, b.w2, 4, g.n1, g.n2, g.n3, g.p2, 6, sw, ty + 2);
    rc |= tma_encode_cubes(&m->u, b.u, 4, g.n1, g.n2, g.n3, g.p2, 1, sw, ty + 1);
    rc |= tma_encode_cubes(&m->q, b.q, 4, g.n1, g.n2, g.n3, g.p2, 1, sw, ty + 1);
    rc |= tma_encode_cubes(&m->s, b.s, 4, g.n1, g.n2, g.n3, g.p2, 1, Lay::TX, ty);
    rc |= tma_encode_cubes(&m->t, b.t, 4, g.n1, g.n2, g.n3, g.p2, 1, Lay::TX, ty);
    rc |= tma_encode_cubes(&m->y3, b.y3, 4, g.n1, g.n2, g.n3, g.p2, 1, Lay::TX, ty + 1);
    return rc ? -3 : 0;
}

namespace {
// bands per CTA for the part's nb updated bands
int part_chunk(const Geom& g, int nb, int chunk) {
    const int tx = (g.n2 + Lay::TX - 1) / Lay::TX, ty = (g.n1 + Lay::TY - 1) / Lay::TY;
    return chunk >= std::min(8, nb) && chunk <= nb ? chunk : tma_chunk(nb, tx * ty);
}
}  // namespace

int k1_tma_part_chunk(const Geom& g, const SlabPart& sp, int chunk) {
    return sp.o1 > sp.o0 ? part_chunk(g, sp.o1 - sp.o0, chunk) : 0;
}

int k1_tma_grid(const Geom& g, const SlabPart& sp, int chunk) {
    const int nb = sp.o1 - sp.o0;
    if (nb <= 0) return 0;
    const int tx = (g.n2 + Lay::TX - 1) / Lay::TX, ty = (g.n1 + Lay::TY - 1) / Lay::TY;
    const int c = part_chunk(g, nb, chunk);
    return tx * ty * ((nb + c - 1) / c);
}

int launch_k1_batch(const BatchCube* cubes, int n, cudaStream_t st) {
    if (n < 1 || n > kBatchMax) return -1;
    static_assert(sizeof(K1BatchTab) <= 32000, "kernel parameter space");
    K1BatchTab t{};
    t.n = n;
    int total = 0;
    for (int c = 0; c < n; ++c) {
        const BatchCube& q = cubes[c];
        const SlabPart whole = whole_cube(q.g);
        K1TArgs& a = t.args[c];
        a.g = q.g;
        a.u_n = (float*)q.b.u_n; a.w1_n = (float*)q.b.w1_n; a.w2_n = (float*)q.b.w2_n;
        a.y1_n = (float*)q.b.y1_n; a.y2_n = (float*)q.b.y2_n;
        a.p = q.p;
        a.sc = q.sc;
        a.l1 = q.l1;
        a.sp = whole;
        a.chunk = part_chunk(q.g, q.g.n3, q.k1_chunk);
        a.hist_fits = a.chunk * Lay::NT <= 65535;
        const int tx = (q.g.n2 + Lay::TX - 1) / Lay::TX, ty = (q.g.n1 + Lay::TY - 1) / Lay::TY;
        const int tz = (q.g.n3 + a.chunk - 1) / a.chunk;
        if (tx > 32767 || ty > 32767 || tz > 32767) return -1;
        t.gx[c] = (short)tx; t.gy[c] = (short)ty; t.gz[c] = (short)tz;
        t.maps[c] = q.maps;
        t.start[c] = total;
        total += tx * ty * tz;
    }
    t.start[n] = total;
    k1_tma_batch<<<total, Lay::NT, Lay::SMEM, st>>>(t);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int k1_batch_configure() {
    const cudaError_t e = cudaFuncSetAttribute(k1_tma_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, Lay::SMEM);
    return e == cudaSuccess ? 0 : -3;
}

int launch_k1_tma(int storage, const Geom& g, const K1Maps& m, const IterBufs& b, const IterParams& p,
                  Scal* sc, const L1Work& w, int chunk, const SlabPart& sp, cudaStream_t st) {
    if (storage != 0) return -1;
    const int nb = sp.o1 - sp.o0;
    if (nb <= 0 || sp.o0 < 0 || sp.o1 > g.n3) return -1;
    K1TArgs a;
    a.g = g;
    a.u_n = (float*)b.u_n; a.w1_n = (float*)b.w1_n; a.w2_n = (float*)b.w2_n;
    a.y1_n = (float*)b.y1_n; a.y2_n = (float*)b.y2_n;
    a.p = p;
    a.sc = sc;
    a.l1 = w;
    a.sp = sp;
    const int tx = (g.n2 + Lay::TX - 1) / Lay::TX, ty = (g.n1 + Lay::TY - 1) / Lay::TY;
    a.chunk = part_chunk(g, nb, chunk);
    // the histogram's packed 16-bit counters hold a CTA's voxels; a split cube
    // passes the longest run of all its launches in sp.max_chunk, so that
    // every launch of the stage agrees
    a.hist_fits = std::max(a.chunk, sp.max_chunk) * Lay::NT <= 65535;
    dim3 grid(tx, ty, (nb + a.chunk - 1) / a.chunk);
    k1_tma<<<grid, Lay::NT, Lay::SMEM, st>>>(m, a);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace gsstv
