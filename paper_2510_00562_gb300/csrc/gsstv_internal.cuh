// Internal definitions shared by the CUDA translation units of libgsstv.
//
// Device layout of one handle (all cubes pitched: element (b, i, j) of a cube
// at offset (b*N1 + i)*P2 + j, P2 = N2 rounded up to 8 so every row starts on
// a 16-byte boundary; the padding columns hold zeros and are never read as
// data):
//   u[2], s[2], t[2], y3[2], q[2]      one cube each, ping-pong by iteration
//   w1[2], w2[2]                       6 cubes each (grid g, component c)
//   y1[2], y2[2]                       2 cubes each (vertical, horizontal)
//   v                                  float32 observation
// y4 is kept as q with a scalar c: y4 = (1 - c) q (the l2-ball step of
// Algorithm 1 is a global rescale, Eq. 23 with Moreau's identity Eq. 3), so
// the scale is applied when y4 is next read instead of in an extra pass.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

namespace gsstv {

// ---------------------------------------------------------------------------
// storage types: iterates are stored as T, every arithmetic step is float32
// ---------------------------------------------------------------------------
template <typename T> struct Store;
template <> struct Store<float> {
    static __device__ __forceinline__ float ld(const float* p) { return *p; }
    static __device__ __forceinline__ void st(float* p, float x) { *p = x; }
};
template <> struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float x) { *p = __float2bfloat16_rn(x); }
};
template <> struct Store<__half> {
    static __device__ __forceinline__ float ld(const __half* p) { return __half2float(*p); }
    static __device__ __forceinline__ void st(__half* p, float x) { *p = __float2half_rn(x); }
};
template <typename T> __device__ __forceinline__ float ldT(const T* p) { return Store<T>::ld(p); }
template <typename T> __device__ __forceinline__ void stT(T* p, float x) { Store<T>::st(p, x); }

// ---------------------------------------------------------------------------
// Stochastic rounding of the 16-bit iterate stores.  With round-to-nearest, a
// 16-bit iterate stops moving once the per-iteration increment of Algorithm 1
// falls below half its last place; rounding up with probability equal to the
// discarded fraction keeps every store unbiased, so small increments still
// accumulate on average.  Random bits: a counter-based stream per voxel and
// iteration -- Wellons' "lowbias32" integer mixer seeds it, a 32-bit LCG
// (Numerical Recipes constants) steps it, and each store takes the high bits.
// The float32 path draws nothing.
// ---------------------------------------------------------------------------
struct SRStream {
    unsigned r;
    __device__ __forceinline__ SRStream(unsigned idx, unsigned iter, unsigned var) {
        unsigned x = idx ^ (iter * 0x9E3779B9u) ^ (var * 0x85EBCA6Bu);
        x ^= x >> 16; x *= 0x7feb352du;
        x ^= x >> 15; x *= 0x846ca68bu;
        x ^= x >> 16;
        r = x;
    }
    __device__ __forceinline__ unsigned next() { r = r * 1664525u + 1013904223u; return r; }
};

template <typename T> struct StoreSR {
    static __device__ __forceinline__ void st(T* p, float x, SRStream&) { stT(p, x); }
};
template <> struct StoreSR<__nv_bfloat16> {
    // bf16 keeps the top 16 bits of the float32 pattern: add 16 random bits
    // below the cut, then truncate (sign-magnitude, so this rounds |x| up with
    // the probability of the discarded fraction)
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float x, SRStream& sr) {
        unsigned u = __float_as_uint(x);
        if ((u & 0x7f800000u) != 0x7f800000u) u += sr.next() >> 16;
        const unsigned short h = (unsigned short)(u >> 16);
        *reinterpret_cast<unsigned short*>(p) = h;
    }
};
template <> struct StoreSR<__half> {
    // fp16 normals keep 10 of the 23 mantissa bits: add 13 random bits below
    // the cut and convert toward zero; tiny values (fp16 subnormals) round to
    // nearest
    static __device__ __forceinline__ void st(__half* p, float x, SRStream& sr) {
        const unsigned u = __float_as_uint(x);
        const unsigned e = u & 0x7f800000u;
        if (e >= 0x38800000u && e != 0x7f800000u)       // |x| >= 2^-14
            *p = __float2half_rz(__uint_as_float(u + (sr.next() >> 19)));
        else
            *p = __float2half_rn(x);
    }
};
template <typename T> __device__ __forceinline__ void stS(T* p, float x, SRStream& sr) { StoreSR<T>::st(p, x, sr); }
template <typename T> constexpr bool kIs16 = !std::is_same<T, float>::value;

// ---------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------
struct Geom {
    int n1, n2, n3;   // rows, columns, bands
    int p2;           // row pitch in elements (multiple of 8)
    long long cube;   // elements of one pitched cube = n3 * n1 * p2
    __host__ __device__ __forceinline__ long long at(int b, int i, int j) const {
        return ((long long)b * n1 + i) * p2 + j;
    }
};

// ---------------------------------------------------------------------------
// l1-ball threshold search state (one per projected vector: 0 = s, 1 = t)
// ---------------------------------------------------------------------------
enum L1Need : int {
    NEED_NONE = 0,      // tau of this iteration is known
    NEED_RADIX0 = 1,    // run the radix histogram, level 0 (bits 30..20)
    NEED_RADIX1 = 2,    // level 1 (bits 19..9) inside the level-0 bin
    NEED_RADIX2 = 3,    // level 2 (bits 8..0): single-value bins
    NEED_GATHER = 4,    // gather the bracket bin and finish with Michelot steps
    NEED_WINDOW = 5,    // one more windowed pass (after a missed window), then radix
};

struct L1Ctl {
    float theta_lo, theta_hi;  // window (theta_lo, theta_hi] for the next pass
    int window_ok;             // 1: K1 accumulates window statistics
    int need;                  // L1Need
    double tau;                // threshold of the current iteration
    double tau_prev;           // threshold of the previous iteration
    double tau_prev2;          // and of the one before
    int have_tau, have_prev, have_prev2;
    double dens;               // candidates per unit of |x| at the last window
    // radix search
    unsigned prefix;           // key bits fixed by the previous levels
    unsigned long long n_above;// elements above the current bracket (exact)
    double s_above;            // their sum (exact up to double rounding)
    float g_lo, g_hi;          // gather window (g_lo, g_hi]
    // K1 histogram of |x| for the next pass (after a miss): bins of the float
    // key >> kHistShift, numbered from hbase; on while hist_left > 0
    unsigned hbase;
    int hist_left;
    long long hits, exact_runs, retry_hits;
};

struct L1Acc {
    unsigned long long n_hi;   // elements with |x| > theta_hi
    double s_hi;               // their sum
    unsigned int m;            // candidates appended (may exceed the capacity)
    unsigned int pad;
};

struct Scal {
    double c[2];               // y4 = (1 - c[p]) q at iteration parity p
    L1Ctl ctl[2];
    L1Acc acc[2];
    double radius[2];          // alpha, beta
    unsigned int k1_ticket, k2_ticket, fb_ticket, g_ticket, w_ticket, pad1;
    int error;                 // bit 0: non-finite norm; bit 1: internal; bit 2: a bounded wait timed out
    int pad0;
    double q2, du2, u2;        // norms of the last K2 pass
    long long iter;
    int done;                  // a batch cube that has stopped (Eq. 28 or its pass cap)
    int stop_parity;           // the parity that holds its state then
    // what the fused pass (TMA-fed K1) counted for vector v, for the finish
    // that follows it: its window statistics and candidates, its histogram
    int k1_win[2], k1_hist[2];
    long long gate_opens;      // passes whose threshold search launches ran (graphs)
    unsigned int fin_ticket;   // CTAs of K1's window finish done (the last sets the search gate)
    unsigned int pad2;
};

constexpr int kHistBins = 2048;        // radix histogram bins per vector
constexpr unsigned kCandCap = 1u << 20; // candidate capacity per vector
constexpr int kNarrowBins = 2048;        // bins of one narrowing round of a candidate list
constexpr double kCandTarget = 65536.0;   // K1's window is sized for at most about this many candidates,
constexpr double kCandTargetWide = 393216.0;  // or this many while the thresholds move fast (histogram on)
constexpr double kRetryTarget = 262144.0; // a retry window after a miss: at most about this many
constexpr unsigned kGatherMax = 1u << 16; // a radix bracket this small is gathered, a larger one refined
// K1's histogram of |x| near the predicted threshold: 1024 bins of 1/256
// octave (the float key >> 15), four octaves, counted in packed 16-bit shared
// counters (so a CTA may count at most 65535 voxels per vector) from a 1/32
// sample of the voxels
constexpr int kHistShift = 15;
constexpr int kK1Bins = 1024;
constexpr int kHistSample = 32;
constexpr int kHistPasses = 6;           // passes the histogram stays on after a miss

// Device workspace of the l1 machinery (shared layout with the standalone
// projection entry point).
struct L1Work {
    float* cand[2];                    // kCandCap floats each
    unsigned long long* hcnt;          // [2][kHistBins]
    unsigned long long* hres;          // [2][kHistBins]
    unsigned long long* k1_n;          // per K1 CTA: [4] counts (window s, t; histogram top s, t)
    double* k1_s;                      // per K1 CTA: [4] sums
    unsigned* khist;                   // [2][kK1Bins] K1 histogram counts (zero between passes)
    // key histogram of each candidate list ([2][3 kNarrowBins]: bin counts, low and
    // high 10 bits of the key residues), filled by the passes that append the
    // candidates and cleared by the finish that reads it; null: not kept
    unsigned* nh;
    unsigned* nbinned;                 // [2] candidates counted into nh
};

// ---------------------------------------------------------------------------
// small numerics helpers
// ---------------------------------------------------------------------------
struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        float y = x - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}
__device__ __forceinline__ unsigned long long warp_sum(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Sum over the block; every thread gets the result.  `buf` holds >= 32 values.
template <typename V>
__device__ __forceinline__ V block_sum(V x, V* buf) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    x = warp_sum(x);
    __syncthreads();
    if (lane == 0) buf[wid] = x;
    __syncthreads();
    V r = (threadIdx.x < (unsigned)nw) ? buf[threadIdx.x] : V(0);
    if (wid == 0) r = warp_sum(r);
    if (threadIdx.x == 0) buf[0] = r;
    __syncthreads();
    r = buf[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ float soft(float x, float tau) {
    float a = fabsf(x) - tau;
    return a > 0.f ? copysignf(a, x) : 0.f;
}

// value of a non-negative float given by its bit pattern, and the size of
// one unit of its last mantissa bit (as double, both exact)
__device__ __forceinline__ double key_value(unsigned key) { return (double)__uint_as_float(key); }
// 2^(e - 150) for the float's biased exponent e (2^-149 for subnormals),
// built as the bit pattern of a double: biased exponent (e - 150) + 1023
__device__ __forceinline__ double key_ulp(unsigned key) {
    const unsigned e = (key >> 23) & 0xffu;
    return __longlong_as_double((long long)((e == 0u ? 1u : e) + 873u) << 52);
}

// Sums over the CTA carried as unevaluated float pairs (hi + lo, Knuth's
// two-sum at every step): FP64 work on this part runs at a small fraction of
// the FP32 rate, so a CTA-wide sum keeps it to thread 0.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void pair_add(float& hi, float& lo, float bhi, float blo) {
    float s, e;
    two_sum(hi, bhi, s, e);
    e = __fadd_rn(e, __fadd_rn(lo, blo));
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}
// The CTA's sum of the threads' compensated sums; the result (a double) is
// valid on thread 0 only.  buf: >= 32 float2 of shared memory.
__device__ __forceinline__ double block_sum_pair(const Kahan& k, float2* buf) {
    float hi = k.s, lo = -k.c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float bh = __shfl_xor_sync(0xffffffffu, hi, o), bl = __shfl_xor_sync(0xffffffffu, lo, o);
        pair_add(hi, lo, bh, bl);
    }
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) buf[w] = make_float2(hi, lo);
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
        float h = buf[0].x, l = buf[0].y;
        for (int k2 = 1; k2 < nw; ++k2) pair_add(h, l, buf[k2].x, buf[k2].y);
        r = (double)h + (double)l;
    }
    return r;
}
// The warp's sum of its lanes' compensated sums as a float pair; every lane
// gets it.
__device__ __forceinline__ void warp_sum_pair(const Kahan& k, float& hi, float& lo) {
    hi = k.s;
    lo = -k.c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float bh = __shfl_xor_sync(0xffffffffu, hi, o), bl = __shfl_xor_sync(0xffffffffu, lo, o);
        pair_add(hi, lo, bh, bl);
    }
}
// Integer sum over the CTA (32-bit lanes, 64-bit result), every thread gets it.
__device__ __forceinline__ unsigned long long block_count(unsigned x, unsigned long long* buf) {
    unsigned long long v = x;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) buf[w] = v;
    __syncthreads();
    unsigned long long r = 0;
    for (int k = 0; k < nw; ++k) r += buf[k];
    __syncthreads();
    return r;
}

// s~ = s - g_s y4 and t~ = t - g_t (D_v^T y3 + y4) of one voxel (the inputs of
// the two l1-ball projections of Algorithm 1), with y4 = cs * q.  Written with
// explicit roundings so that every kernel that needs them (the stencil pass,
// the radix search and the light pass) computes bit-identical values.
__device__ __forceinline__ void s_t_tilde(float s, float t, float y3, float y3_up, float q, float cs,
                                          int i, int n1, float gs, float gt, float& xs, float& xt) {
    const float y4 = __fmul_rn(cs, q);
    xs = __fsub_rn(s, __fmul_rn(gs, y4));
    const float dvt = __fsub_rn(y3_up, i <= n1 - 2 ? y3 : 0.f);
    xt = __fsub_rn(t, __fmul_rn(gt, __fadd_rn(dvt, y4)));
}

// ---------------------------------------------------------------------------
// window accounting for one |x| value, used by K1 and by the gather pass
// ---------------------------------------------------------------------------
struct WinAcc {
    unsigned long long n = 0;
    Kahan s;
};

// Appends the lanes' candidates with one atomic per warp.
__device__ __forceinline__ void append_candidate(bool take, float x, float* cand, unsigned* cnt) {
    unsigned mask = __ballot_sync(0xffffffffu, take);
    if (mask == 0) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(cnt, (unsigned)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (take) {
        unsigned k = base + __popc(mask & ((1u << lane) - 1u));
        if (k < kCandCap) cand[k] = x;
    }
}

// ---------------------------------------------------------------------------
// kernel launchers (host)
// ---------------------------------------------------------------------------
// Streaming multiprocessors of the current device, queried once per device
// (grids are sized in multiples of it).
int device_sms();

struct IterBufs {
    // current (read) and next (write) buffers of one iteration parity
    const void *u, *s, *t, *y3, *q, *w1, *w2, *y1, *y2;
    void *u_n, *s_n, *t_n, *y3_n, *q_n, *w1_n, *w2_n, *y1_n, *y2_n;
    const float* v;
};

struct IterParams {
    float gamma_u, gamma_w1, gamma_w2, gamma_s, gamma_t;
    float gamma_y1, gamma_y2, gamma_y3, gamma_y4;
    float thr_w1, thr_w2;        // gamma_w1 * omega, gamma_w2
    float mu_lo, mu_hi;
    double eps;
    int parity;                  // iteration parity (selects c[])
    int tau_exact;               // 1: skip the window statistics
    // the stopping rule applied on the device (batch cubes; max_iter = 0: off)
    int max_iter;
    int check_every;
    double tol;
    int* live;                   // counter of the batch's unfinished cubes
};

// Tensor maps over the current-parity buffers read by the TMA-fed K1.
struct K1Maps {
    CUtensorMap y1, y2, w1, w2, u, q, s, t, y3;
};

// The bands one launch updates when a cube is stored as band slabs in
// separate allocations (only D_s couples bands, Sec. II-A, so a slab needs one
// halo band on each side).  The launch's storage holds bands [band0, band0 +
// g.n3) of a cube of n3g bands, and the launch updates the stored bands
// [o0, o1).  Every global sum of a pass stage (the l2-ball norm, the Eq. 28
// norms, the l1 threshold statistics) is finished once for all the stage's
// launches (by the last of their CTAs, or by a finishing launch after them):
// this launch's CTAs are numbered from cta_base among cta_total.  The whole
// cube in one launch: whole_cube(g).
struct SlabPart {
    int band0 = 0, n3g = 0, o0 = 0, o1 = 0;
    int cta_base = 0, cta_total = 0;     // cta_total = 0: this launch alone
    int max_chunk = 0;                   // K1: the longest band run of any launch of the stage
};
inline SlabPart whole_cube(const Geom& g) {
    SlabPart s;
    s.n3g = g.n3;
    s.o1 = g.n3;
    return s;
}

int k1_tma_ctas(const Geom& g);
int k1_tma_chunk_candidates(const Geom& g, int* out, int cap);
int k1_tma_configure(int storage);
int k1_tma_maps(int storage, const Geom& g, const IterBufs& b, K1Maps* m);
// CTAs of one K1 launch over the part's bands, and its bands per CTA (chunk
// as for launch_k1_tma)
int k1_tma_grid(const Geom& g, const SlabPart& sp, int chunk);
int k1_tma_part_chunk(const Geom& g, const SlabPart& sp, int chunk);
// chunk: bands per CTA (0 or out of range: the wave/prologue model's choice)
int launch_k1_tma(int storage, const Geom& g, const K1Maps& m, const IterBufs& b, const IterParams& p,
                  Scal* sc, const L1Work& w, int chunk, const SlabPart& sp, cudaStream_t st);

int launch_k1(int storage, const Geom& g, const IterBufs& b, const IterParams& p, Scal* sc,
              const L1Work& w, int n_cta_slots, cudaStream_t st);
int k1_grid_ctas(const Geom& g);
int k1_configure(int storage);
int light_configure(int storage);
// CTAs of one launch of the threshold passes and of K2 over the part's bands
int window_grid(const Geom& g, const SlabPart& sp, int part_cap);
int radix_grid(const Geom& g, const SlabPart& sp);
int gather_grid(const Geom& g, const SlabPart& sp);
int k2_grid(const Geom& g, const SlabPart& sp, int part_cap);
int launch_fallback(int storage, int level, const Geom& g, const IterBufs& b, const IterParams& p,
                    Scal* sc, const L1Work& w, const SlabPart& sp, cudaStream_t st);
int launch_gather(int storage, const Geom& g, const IterBufs& b, const IterParams& p, Scal* sc,
                  const L1Work& w, const SlabPart& sp, cudaStream_t st);
int launch_window(int storage, const Geom& g, const IterBufs& b, const IterParams& p, Scal* sc,
                  const L1Work& w, int part_cap, const SlabPart& sp, cudaStream_t st);
int launch_k2(int storage, const Geom& g, const IterBufs& b, const IterParams& p, Scal* sc,
              double* part, int part_cap, const SlabPart& sp, cudaStream_t st);
// Sets `cond` (a graph conditional handle) to whether any of the n cubes
// whose scalars are sc[] needs a threshold search after K1's finish (for the
// cooperative K1, whose last CTA finishes its windows itself).
int launch_search_gate(Scal* const* sc, int n, cudaGraphConditionalHandle cond, cudaStream_t st);
// The finish of K1's windows (mode 2; parts: K1's CTAs, four partials each in
// pn / ps), of the retry window (mode 0; parts: CTAs of the window pass(es),
// their partial sums in pn / ps) or of the gathered radix bracket (mode 1),
// for every vector that needs it: one launch after the pass(es) it finishes.
// gated (mode 2 in a graph): its last CTA also sets `cond` to whether a
// threshold search is still needed.
int launch_search_finish(int mode, Scal* sc, const L1Work& w, int nvec, const unsigned long long* pn,
                         const double* ps, int parts, cudaStream_t st, int gated = 0,
                         cudaGraphConditionalHandle cond = 0);
int k2_grid_ctas(const Geom& g);

// ---------------------------------------------------------------------------
// batches: every stage of a pass launched once for many independent cubes
// ---------------------------------------------------------------------------
// What a batch launch needs of one cube at one iteration parity.  Each cube
// keeps its own state, reductions and stopping rule (IterParams max_iter, tol,
// check_every: K2 sets Scal::done on the device); a launch covers the CTAs of
// every cube, each CTA finds its cube in a table of first CTAs, and the CTAs
// of a cube that is done return at once.  Float32 storage.
constexpr int kBatchMax = 64;
struct BatchCube {
    Geom g;
    IterBufs b;
    IterParams p;
    Scal* sc;
    L1Work l1;
    double* k2_part;
    int k2_cap;
    int k1_chunk;            // bands per K1 CTA (as the cube's handle runs it)
    int k1_ctas;             // capacity of the cube's per-CTA statistics
    const K1Maps* maps;      // the cube's tensor maps at this parity (device memory)
};
// Each launches one stage for cubes[0..n) on st (n <= kBatchMax).
int launch_k1_batch(const BatchCube* cubes, int n, cudaStream_t st);
int launch_window_batch(const BatchCube* cubes, int n, cudaStream_t st);
int launch_radix_batch(const BatchCube* cubes, int n, int level, cudaStream_t st);
int launch_gather_batch(const BatchCube* cubes, int n, cudaStream_t st);
int launch_finish_batch(const BatchCube* cubes, int n, int mode, cudaStream_t st, int gated = 0,
                        cudaGraphConditionalHandle cond = 0);
int launch_k2_batch(const BatchCube* cubes, int n, cudaStream_t st);
int batch_configure();

// float32 cubes between two layouts: ncubes cubes of nbands x n1 rows of n2
// values, source and destination each with its own row pitch and cube stride
// (in floats); y4 = (1 - *scale) q when scale is not NULL
int launch_copy_f32(const float* src, long long src_pitch, long long src_cube, float* dst, long long dst_pitch,
                    long long dst_cube, int n1, int n2, int nbands, int ncubes, const double* scale,
                    cudaStream_t st);

// state conversion (float32 views <-> pitched storage)
int launch_pack(int storage, const float* src, void* dst, const Geom& g, int ncubes, cudaStream_t st);
int launch_pitched_to_storage(int storage, const float* src, void* dst, const Geom& g, cudaStream_t st);
int launch_dense_to_pitched(const float* src, float* dst, const Geom& g, cudaStream_t st);
int launch_unpack(int storage, const void* src, float* dst, const Geom& g, int ncubes, cudaStream_t st);
// a whole state (u, s, t, w1, w2, y1, y2, y3, and y4 = (1 - *c) q) in one
// launch; returns 1 when the storage or the row geometry does not allow it
int launch_unpack_state(int storage, const void* const src[9], float* const dst[9], const double* c,
                        const Geom& g, cudaStream_t st);
int launch_scale_unpack(int storage, const void* q, const double* c, float* dst, const Geom& g,
                        cudaStream_t st);

// reverse mode of one pass on dense float32 states (k_adjoint.cu).  x, x1:
// states k and k+1 (u, s, t, w1, w2, y1, y2, y3, y4); b1: adjoint of state
// k+1; bo: adjoint of state k (may be b1 itself); v with row pitch v_pitch;
// vbar += the adjoint of v; pbar[0..3] += those of eps, alpha, beta, omega.
// prm: g_u, g_w1, g_w2, g_s, g_t, g_y1..g_y4, thr_w1, thr_w2, mu_lo, mu_hi,
// eps, alpha, beta.  work: adjoint_workspace_bytes(N) bytes.
// Regions of the reverse mode's scratch start on 256-byte boundaries: a cube
// of n floats takes adj_stride(n) floats (the global sums are doubles).
inline long long adj_stride(long long n) { return (n + 63) / 64 * 64; }
size_t adjoint_workspace_bytes(long long n);
int launch_adjoint_step(int n1, int n2, int n3, const float* const x[9], const float* const x1[9],
                        const float* const b1[9], float* const bo[9], const float* v, int v_pitch,
                        float* vbar, double* pbar, void* work, const double prm[16], cudaStream_t st);
// y += a x on n floats
int launch_axpy(float* y, const float* x, float a, long long n, cudaStream_t st);

// standalone projection
int l1_project_standalone(const float* x, long long n, double radius, float* out, double* tau,
                          cudaStream_t st);

}  // namespace gsstv
