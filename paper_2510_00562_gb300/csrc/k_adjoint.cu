// Reverse mode of one pass of Algorithm 1 (a vector-Jacobian product), for
// gradients of losses of the unrolled iteration.
//
// Forward pass (state x = (u, s, t, w1, w2, y1..y4), observation v):
//   a_u = u - g_u (D^T y1 + D_s^T D^T y2 + y4),   u+ = box(a_u)       (Eq. 21)
//   a_wk = wk + g_wk L yk,                         wk+ = S_thk(a_wk)    (Eq. 24)
//   a_s = s - g_s y4,  a_t = t - g_t (D_v^T y3 + y4),  s+, t+ = l1-ball projections
//   x' = 2 x+ - x
//   y1+ = y1 + g1 (D u' - L^T w1'),  y2+ = y2 + g2 (D D_s u' - L^T w2')
//   y3+ = y3 + g3 D_v t',  q = y4 + g4 (u' + s' + t') - g4 v,  y4+ = (1 - c) q,
//   c = min(1, eps g4 / ||q||)                                          (Eq. 23)
// The transpose runs these steps backwards with the derivatives that hold
// almost everywhere: the box passes where mu_lo < u+ < mu_hi; the group
// shrink of x with threshold th has Jacobian (1 - th/|x|) I + th x x^T/|x|^3
// above the threshold (derivative -x/|x| in th) and 0 below; the l1-ball
// projection is the identity inside the ball and, outside, keeps the active
// set A = {s+ != 0} with adjoint p - sign S/|A|, S = sum_A sign p (derivative
// S/|A| in the radius); the l2 step has Jacobian I - (eps g4/|q|)(I - q^ q^^T)
// for |q| > eps g4 (derivative -g4 q^ . in eps) and 0 otherwise.
//
// All arrays are dense C-contiguous float32: cubes (N3, N1, N2), dual pairs
// (2, N3, N1, N2) (vertical at (i+1/2, j), horizontal at (i, j+1/2)), the
// auxiliary w (3, 2, N3, N1, N2) (grids (i+1/2, j), (i, j+1/2), (i, j)).
// D, D_s are forward differences with Neumann boundary; L reads the dual pair
// masked where D is structurally zero (vertical component on the last row,
// horizontal component on the last column), its grid-(i+1/2, j) output is
// zero on the last row and its grid-(i, j+1/2) output zero on the last
// column; L^T is its exact transpose.
//
// Five launches on 32 x 8 thread blocks (32 columns x 8 rows of one band,
// persistent over the rows; 4 blocks per SM), a few device doubles for the
// global sums, nothing synchronises the host.  In each voxel's body the
// loads of buffers that the kernel also writes (the adjoint, in place) come
// before every store; everything else is read through the read-only path,
// so the compiler may issue those loads early:
//   SUMS  |q|^2, q . y4_bar, |a_s|_1, |a_t|_1 (the l2 step and whether each
//         l1 ball is active);
//   CUBE  the l2 step, the transposed dual ascents and extrapolations of u,
//         s, t, the box; sums for the l1 adjoints;
//   AUX   the group-shrink adjoints of w1, w2 (independent of CUBE);
//   FIN1  the l1 adjoints and the transposed operators onto y3, y4;
//   FIN2  the transposed operators onto y1, y2.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "gsstv_internal.cuh"

namespace gsstv {
namespace {

constexpr int BX = 32, BY = 8, NTA = BX * BY;

struct Dims {
    int n1, n2, n3;
    int vp;                                       // row pitch of v (floats)
    int rows;                                     // n3 * n1
    long long plane;                              // n1 * n2
    long long N;                                  // voxels
};

struct SV {
    const float *u, *s, *t, *w1, *w2, *y1, *y2, *y3, *y4;
};
struct SW {
    float *u, *s, *t, *w1, *w2, *y1, *y2, *y3, *y4;
};

// scalars of one reverse pass (doubles on the device)
enum { QQ = 0, QB, L1S, L1T, SS, NS, ST, NT_, TH1, NSCAL };

struct AdjArgs {
    Dims d;
    SV x, x1, b1;                 // state k, state k+1, adjoint of state k+1
    SW b;                         // adjoint of state k (written; may be b1)
    int inplace;                  // b and b1 are the same buffers
    const float* v;
    float* vbar;                  // += adjoint of v
    double* pbar;                 // += adjoints of eps, alpha, beta, omega
    double* sc;                   // NSCAL scalars, zeroed before the pass
    float *gbar, *aw1, *aw2, *s1b, *t1b;   // temporaries (N, 6N, 6N, N, N)
    float g_u, g_w1, g_w2, g_s, g_t, g1, g2, g3, g4, th1, th2, mu_lo, mu_hi;
    double eps, alpha, beta, g4d, g_w1d;
};

// read-only data (states k, k+1 and v; never written during a pass)
__device__ __forceinline__ float rd(const float* p, long long k) { return __ldg(p + k); }

// ---- stencils on dense cubes (value at voxel l = (b, i, j) of an operator's
// output).  They read through the read-only path: every kernel applies them
// only to arrays that no thread writes while it runs.  IN = the voxel is
// interior in its band (1 <= i <= N1-2, 1 <= j <= N2-2): then every spatial
// neighbour they touch exists and no boundary mask applies, so the checks
// are compiled out; the band neighbours are checked either way.

// p at (b, i+di, j+dj), zero outside the image
template <bool IN>
__device__ __forceinline__ float nb(const float* p, const Dims& d, long long l, int i, int j, int di, int dj) {
    if (!IN && (i + di < 0 || i + di >= d.n1 || j + dj < 0 || j + dj >= d.n2)) return 0.f;
    return rd(p, l + (long long)di * d.n2 + dj);
}
// D_v x, D_h x
template <bool IN>
__device__ __forceinline__ float dv(const float* x, const Dims& d, long long l, int i) {
    return (IN || i < d.n1 - 1) ? rd(x, l + d.n2) - rd(x, l) : 0.f;
}
template <bool IN>
__device__ __forceinline__ float dh(const float* x, const Dims& d, long long l, int j) {
    return (IN || j < d.n2 - 1) ? rd(x, l + 1) - rd(x, l) : 0.f;
}
// transposes: (D_v^T y)(i) = y(i-1) [i >= 1] - y(i) [i <= N1-2]
template <bool IN>
__device__ __forceinline__ float dvT(const float* y, const Dims& d, long long l, int i) {
    float r = 0.f;
    if (IN || i >= 1) r += rd(y, l - d.n2);
    if (IN || i <= d.n1 - 2) r -= rd(y, l);
    return r;
}
template <bool IN>
__device__ __forceinline__ float dhT(const float* y, const Dims& d, long long l, int j) {
    float r = 0.f;
    if (IN || j >= 1) r += rd(y, l - 1);
    if (IN || j <= d.n2 - 2) r -= rd(y, l);
    return r;
}
// D^T y for a dual pair y (2 planes of N)
template <bool IN>
__device__ __forceinline__ float dT(const float* y, const Dims& d, long long l, int i, int j) {
    return dvT<IN>(y, d, l, i) + dhT<IN>(y + d.N, d, l, j);
}
// (D_s^T D^T y)(b) = (D^T y)(b-1) [b >= 1] - (D^T y)(b) [b <= N3-2]
template <bool IN>
__device__ __forceinline__ float dsT_dT(const float* y, const Dims& d, long long l, int b, int i, int j) {
    float r = 0.f;
    if (b >= 1) r += dT<IN>(y, d, l - d.plane, i, j);
    if (b <= d.n3 - 2) r -= dT<IN>(y, d, l, i, j);
    return r;
}
// dual-pair entries read by L, masked where D is structurally zero
template <bool IN>
__device__ __forceinline__ float yvm(const float* y, const Dims& d, long long l, int i, int j, int di, int dj) {
    if (!IN && !(i + di >= 0 && i + di < d.n1 - 1 && j + dj >= 0 && j + dj < d.n2)) return 0.f;
    return rd(y, l + (long long)di * d.n2 + dj);
}
template <bool IN>
__device__ __forceinline__ float yhm(const float* y, const Dims& d, long long l, int i, int j, int di, int dj) {
    if (!IN && !(i + di >= 0 && i + di < d.n1 && j + dj >= 0 && j + dj < d.n2 - 1)) return 0.f;
    return rd(y, d.N + l + (long long)di * d.n2 + dj);
}
// L y: out[k], k = 2 g + c (g grid, c = vertical / horizontal)
template <bool IN>
__device__ __forceinline__ void Lop(const float* y, const Dims& d, long long l, int i, int j, float out[6]) {
    const float v00 = yvm<IN>(y, d, l, i, j, 0, 0), vm0 = yvm<IN>(y, d, l, i, j, -1, 0),
                v01 = yvm<IN>(y, d, l, i, j, 0, 1), vm1 = yvm<IN>(y, d, l, i, j, -1, 1);
    const float h00 = yhm<IN>(y, d, l, i, j, 0, 0), h0m = yhm<IN>(y, d, l, i, j, 0, -1),
                h10 = yhm<IN>(y, d, l, i, j, 1, 0), h1m = yhm<IN>(y, d, l, i, j, 1, -1);
    const bool mv = IN || i < d.n1 - 1, mh = IN || j < d.n2 - 1;
    out[0] = mv ? v00 : 0.f;
    out[1] = mv ? 0.25f * (h00 + h0m + h10 + h1m) : 0.f;
    out[2] = mh ? 0.25f * (v00 + vm0 + v01 + vm1) : 0.f;
    out[3] = mh ? h00 : 0.f;
    out[4] = 0.5f * (v00 + vm0);
    out[5] = 0.5f * (h00 + h0m);
}
// component k of w at (b, i+di, j+dj), zero outside the image and where L's
// output is structurally zero (grid 0 on the last row, grid 1 on the last column)
template <bool IN>
__device__ __forceinline__ float wk(const float* w, const Dims& d, int k, long long l, int i, int j, int di, int dj) {
    if (!IN) {
        const int ii = i + di, jj = j + dj;
        if (ii < 0 || ii >= d.n1 || jj < 0 || jj >= d.n2) return 0.f;
        if (k < 2 && ii == d.n1 - 1) return 0.f;
        if ((k == 2 || k == 3) && jj == d.n2 - 1) return 0.f;
    }
    return rd(w, (long long)k * d.N + l + (long long)di * d.n2 + dj);
}
// L^T w: (vertical, horizontal)
template <bool IN>
__device__ __forceinline__ void LTop(const float* w, const Dims& d, long long l, int i, int j, float& gv, float& gh) {
    const bool mv = IN || i < d.n1 - 1, mh = IN || j < d.n2 - 1;
    gv = mv ? (wk<IN>(w, d, 0, l, i, j, 0, 0) +
               0.25f * (wk<IN>(w, d, 2, l, i, j, 0, 0) + wk<IN>(w, d, 2, l, i, j, 1, 0) +
                        wk<IN>(w, d, 2, l, i, j, 0, -1) + wk<IN>(w, d, 2, l, i, j, 1, -1)) +
               0.5f * (wk<IN>(w, d, 4, l, i, j, 0, 0) + wk<IN>(w, d, 4, l, i, j, 1, 0)))
            : 0.f;
    gh = mh ? (0.25f * (wk<IN>(w, d, 1, l, i, j, 0, 0) + wk<IN>(w, d, 1, l, i, j, 0, 1) +
                        wk<IN>(w, d, 1, l, i, j, -1, 0) + wk<IN>(w, d, 1, l, i, j, -1, 1)) +
               wk<IN>(w, d, 3, l, i, j, 0, 0) +
               0.5f * (wk<IN>(w, d, 5, l, i, j, 0, 0) + wk<IN>(w, d, 5, l, i, j, 0, 1)))
            : 0.f;
}

// Sum over the block of 32 x 8 threads (valid on thread (0, 0)).
__device__ __forceinline__ double block_sum_d(double x, double* buf) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    __syncthreads();
    if (threadIdx.x == 0) buf[threadIdx.y] = x;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0 && threadIdx.y == 0)
        for (int k = 0; k < BY; ++k) r += buf[k];
    return r;
}

// The voxels of this thread: column j of the block, rows (b*N1 + i) strided
// by the grid; body(b, i, j, l, interior) per voxel, interior a
// std::integral_constant<bool, ...> selecting the unchecked stencils.  The
// choice is made per warp (one row, 32 columns): a warp with a border voxel
// takes the checked path for all its lanes, so no warp runs both.
template <int UNROLL = 1, class F>
__device__ __forceinline__ void for_voxels(const Dims& d, F&& body) {
    const int j = blockIdx.x * BX + threadIdx.x;
    if (j >= d.n2) return;
    const unsigned lanes = __activemask();          // the same lanes in every iteration
    const bool jin = j >= 1 && j <= d.n2 - 2;
#pragma unroll UNROLL
    for (int row = blockIdx.y * BY + threadIdx.y; row < d.rows; row += gridDim.y * BY) {
        const int b = row / d.n1, i = row - b * d.n1;
        const long long l = (long long)row * d.n2 + j;
        if (__all_sync(lanes, jin && i >= 1 && i <= d.n1 - 2))
            body(b, i, j, l, std::true_type{});
        else
            body(b, i, j, l, std::false_type{});
    }
}

// Float partial sums over a thread's voxels, moved into doubles every 32
// terms: FP64 issue is scarce on this part, float alone drifts over
// hundreds of terms.
template <int K>
struct Partial {
    float f[K];
    double d[K];
    int n;
    __device__ __forceinline__ Partial() : n(0) {
#pragma unroll
        for (int k = 0; k < K; ++k) { f[k] = 0.f; d[k] = 0.0; }
    }
    __device__ __forceinline__ void step() {
        if (++n == 32) flush();
    }
    __device__ __forceinline__ void flush() {
#pragma unroll
        for (int k = 0; k < K; ++k) { d[k] += (double)f[k]; f[k] = 0.f; }
        n = 0;
    }
};

// q = y4 + g4 (u' + s' + t') - g4 v at voxel l = (b, i, j)
__device__ __forceinline__ float q_at(const AdjArgs& a, long long l, int b, int i, int j) {
    const float up = 2.f * rd(a.x1.u, l) - rd(a.x.u, l), sp = 2.f * rd(a.x1.s, l) - rd(a.x.s, l),
                tp = 2.f * rd(a.x1.t, l) - rd(a.x.t, l);
    const float v = rd(a.v, ((long long)b * a.d.n1 + i) * a.d.vp + j);
    return rd(a.x.y4, l) + a.g4 * (up + sp + tp) - a.g4 * v;
}

// SUMS: |q|^2, q . y4_bar+, |a_s|_1, |a_t|_1
__global__ void __launch_bounds__(NTA, 4) k_adj_sums(const AdjArgs a) {
    __shared__ double buf[BY];
    Partial<4> p;
    for_voxels<2>(a.d, [&](int b, int i, int j, long long l, auto in) {
        constexpr bool IN = decltype(in)::value;
        (void)b;
        const float q = q_at(a, l, b, i, j);
        const float y4 = rd(a.x.y4, l);
        p.f[0] = fmaf(q, q, p.f[0]);
        p.f[1] = fmaf(q, rd(a.b1.y4, l), p.f[1]);
        p.f[2] += fabsf(rd(a.x.s, l) - a.g_s * y4);
        p.f[3] += fabsf(rd(a.x.t, l) - a.g_t * (dvT<IN>(a.x.y3, a.d, l, i) + y4));
        p.step();
    });
    p.flush();
    const double r0 = block_sum_d(p.d[0], buf), r1 = block_sum_d(p.d[1], buf), r2 = block_sum_d(p.d[2], buf),
                 r3 = block_sum_d(p.d[3], buf);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        atomicAdd(a.sc + QQ, r0);
        atomicAdd(a.sc + QB, r1);
        atomicAdd(a.sc + L1S, r2);
        atomicAdd(a.sc + L1T, r3);
    }
}

// CUBE: l2 step, transposed dual ascents, extrapolations of u, s, t, box;
// sums for the l1 adjoints
__global__ void __launch_bounds__(NTA, 4) k_adj_cube(const AdjArgs a) {
    __shared__ double buf[BY];
    __shared__ float scal[3];
    const Dims& d = a.d;
    const long long N = d.N;
    // the l2 step's scalars, once per block (FP64 issue is scarce)
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const double nq = sqrt(a.sc[QQ]);
        const bool act = nq > a.eps * a.g4d;
        const double qdot = act ? a.sc[QB] / nq : 0.0;          // q^ . y4_bar+
        scal[0] = act ? 1.f : 0.f;
        scal[1] = act ? (float)(a.eps * a.g4d / nq) : 0.f;
        scal[2] = act ? (float)(qdot / nq) : 0.f;               // (q^ . y4_bar+) / |q|
        if (act && blockIdx.x == 0 && blockIdx.y == 0) atomicAdd(a.pbar + 0, -a.g4d * qdot);
    }
    __syncthreads();
    const bool l2act = scal[0] != 0.f;
    const float fk = scal[1], qs = scal[2];
    Partial<2> p;
    unsigned ns = 0, nt = 0;
    for_voxels(d, [&](int b, int i, int j, long long l, auto in) {
        constexpr bool IN = decltype(in)::value;
        // loads of the buffers that this kernel also writes (in place), first
        const float y4b = a.b1.y4[l], bu = a.b1.u[l], bs = a.b1.s[l], bt = a.b1.t[l], vb = a.vbar[l];
        // y4+ = (1 - c) q
        const float qbar = l2act ? y4b - fk * (y4b - q_at(a, l, b, i, j) * qs) : 0.f;
        const float ub_ = a.g4 * qbar + a.g2 * dsT_dT<IN>(a.b1.y2, d, l, b, i, j) + a.g1 * dT<IN>(a.b1.y1, d, l, i, j);
        const float sb_ = a.g4 * qbar;
        const float tb_ = a.g4 * qbar + a.g3 * dvT<IN>(a.b1.y3, d, l, i);
        // u+ = box(a_u): the adjoint passes where mu_lo < u+ < mu_hi
        const float u1 = rd(a.x1.u, l);
        const float u1bar = bu + 2.f * ub_;
        const float aub = (u1 > a.mu_lo && u1 < a.mu_hi) ? u1bar : 0.f;
        const float s1bar = bs + 2.f * sb_, t1bar = bt + 2.f * tb_;
        if (!a.inplace) {
            const float c0 = rd(a.b1.y1, l), c1 = rd(a.b1.y1, N + l), c2 = rd(a.b1.y2, l),
                        c3 = rd(a.b1.y2, N + l), c4 = rd(a.b1.y3, l);
            a.b.y1[l] = c0;
            a.b.y1[N + l] = c1;
            a.b.y2[l] = c2;
            a.b.y2[N + l] = c3;
            a.b.y3[l] = c4;
        }
        a.vbar[l] = vb - a.g4 * qbar;
        a.b.u[l] = -ub_ + aub;
        a.gbar[l] = -a.g_u * aub;
        a.s1b[l] = s1bar;
        a.t1b[l] = t1bar;
        a.b.s[l] = -sb_;
        a.b.t[l] = -tb_;
        a.b.y4[l] = qbar;
        const float s1 = rd(a.x1.s, l), t1 = rd(a.x1.t, l);
        if (s1 != 0.f) { p.f[0] += (s1 > 0.f ? s1bar : -s1bar); ++ns; }
        if (t1 != 0.f) { p.f[1] += (t1 > 0.f ? t1bar : -t1bar); ++nt; }
        p.step();
    });
    p.flush();
    const double r0 = block_sum_d(p.d[0], buf), r1 = block_sum_d((double)ns, buf),
                 r2 = block_sum_d(p.d[1], buf), r3 = block_sum_d((double)nt, buf);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        atomicAdd(a.sc + SS, r0);
        atomicAdd(a.sc + NS, r1);
        atomicAdd(a.sc + ST, r2);
        atomicAdd(a.sc + NT_, r3);
    }
}

// AUX: w+ = S(a_w), a_w = w + g L y, group shrink with threshold th; the
// adjoint of w' is -g_y L y_bar+ (from the dual ascent), that of w+ is
// w+_bar + 2 w'_bar
__global__ void __launch_bounds__(NTA, 4) k_adj_aux(const AdjArgs a) {
    __shared__ double buf[BY];
    const Dims& d = a.d;
    const long long N = d.N;
    Partial<1> p;
    for_voxels(d, [&](int b, int i, int j, long long l, auto in) {
        constexpr bool IN = decltype(in)::value;
        // the adjoints of w1+, w2+ (this kernel overwrites them in place), first
        float pw[12];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            pw[k] = a.b1.w1[(long long)k * N + l];
            pw[6 + k] = a.b1.w2[(long long)k * N + l];
        }
#pragma unroll
        for (int set = 0; set < 2; ++set) {
            const float* w = set ? a.x.w2 : a.x.w1;
            float* bw = set ? a.b.w2 : a.b.w1;
            float* aw = set ? a.aw2 : a.aw1;
            const float gw = set ? a.g_w2 : a.g_w1;
            const float gy = set ? a.g2 : a.g1;
            const float thr = set ? a.th2 : a.th1;
            float lw[6], ly[6];
            Lop<IN>(set ? a.b1.y2 : a.b1.y1, d, l, i, j, lw);
            Lop<IN>(set ? a.x.y2 : a.x.y1, d, l, i, j, ly);
#pragma unroll
            for (int g = 0; g < 3; ++g) {
                const long long kv = (long long)(2 * g) * N + l, kh = (long long)(2 * g + 1) * N + l;
                const float xv = rd(w, kv) + gw * ly[2 * g], xh = rd(w, kh) + gw * ly[2 * g + 1];
                const float wbv = -gy * lw[2 * g], wbh = -gy * lw[2 * g + 1];     // adjoint of w'
                const float pv = pw[6 * set + 2 * g] + 2.f * wbv;                   // total of w+
                const float ph = pw[6 * set + 2 * g + 1] + 2.f * wbh;
                const float n = sqrtf(xv * xv + xh * xh);
                float av = 0.f, ah = 0.f;
                if (n > thr) {
                    const float rn = 1.f / n;
                    const float xhv = xv * rn, xhh = xh * rn;
                    const float dot = xhv * pv + xhh * ph;
                    const float k2 = thr * rn, k1 = 1.f - k2;
                    av = k1 * pv + k2 * xhv * dot;
                    ah = k1 * ph + k2 * xhh * dot;
                    if (set == 0) p.f[0] -= dot;
                }
                aw[kv] = av;
                aw[kh] = ah;
                bw[kv] = -wbv + av;
                bw[kh] = -wbh + ah;
            }
        }
        p.step();
    });
    p.flush();
    const double r0 = block_sum_d(p.d[0], buf);
    if (threadIdx.x == 0 && threadIdx.y == 0) atomicAdd(a.sc + TH1, r0);
}

// FIN1: the l1 adjoints; y4 and y3
__global__ void __launch_bounds__(NTA, 4) k_adj_fin1(const AdjArgs a) {
    __shared__ float scal[4];
    const Dims& d = a.d;
    // the l1 adjoints' scalars, once per block
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const bool is = a.sc[L1S] <= a.alpha, it = a.sc[L1T] <= a.beta;
        const double ksd = (!is && a.sc[NS] > 0) ? a.sc[SS] / a.sc[NS] : 0.0;
        const double ktd = (!it && a.sc[NT_] > 0) ? a.sc[ST] / a.sc[NT_] : 0.0;
        scal[0] = is ? 1.f : 0.f;
        scal[1] = it ? 1.f : 0.f;
        scal[2] = (float)ksd;
        scal[3] = (float)ktd;
        if (blockIdx.x == 0 && blockIdx.y == 0) {
            if (!is) atomicAdd(a.pbar + 1, ksd);
            if (!it) atomicAdd(a.pbar + 2, ktd);
            atomicAdd(a.pbar + 3, a.g_w1d * a.sc[TH1]);
        }
    }
    __syncthreads();
    const bool in_s = scal[0] != 0.f, in_t = scal[1] != 0.f;
    const float ks = scal[2], kt = scal[3];
    // adjoint of t~ = t - g_t (D_v^T y3 + y4) at voxel l (pointwise in CUBE's
    // outputs, which no thread writes here)
    auto atb_at = [&](long long l) {
        const float t1 = rd(a.x1.t, l), tb = rd(a.t1b, l);
        return in_t ? tb : (t1 != 0.f ? tb - (t1 > 0.f ? kt : -kt) : 0.f);
    };
    for_voxels(d, [&](int b, int i, int j, long long l, auto in) {
        (void)b; (void)j; (void)in;                 // pointwise (no stencils)
        // the adjoint entries updated here, first
        const float bs = a.b.s[l], bt = a.b.t[l], b4 = a.b.y4[l], b3 = a.b.y3[l];
        const float s1 = rd(a.x1.s, l), s1b = rd(a.s1b, l);
        const float asb = in_s ? s1b : (s1 != 0.f ? s1b - (s1 > 0.f ? ks : -ks) : 0.f);
        const float atb = atb_at(l);
        const float gb = rd(a.gbar, l);
        // y3 -= g_t D_v a_t_bar
        const float dvat = i < d.n1 - 1 ? atb_at(l + d.n2) - atb : 0.f;
        a.b.s[l] = bs + asb;
        a.b.t[l] = bt + atb;
        a.b.y4[l] = b4 + (gb - a.g_s * asb - a.g_t * atb);
        a.b.y3[l] = b3 - a.g_t * dvat;
    });
}

// FIN2: y1 += D G_bar + g_w1 L^T aw1;  y2 += D D_s G_bar + g_w2 L^T aw2
__global__ void __launch_bounds__(NTA, 4) k_adj_fin2(const AdjArgs a) {
    const Dims& d = a.d;
    const long long N = d.N;
    for_voxels(d, [&](int b, int i, int j, long long l, auto in) {
        constexpr bool IN = decltype(in)::value;
        // the adjoint entries updated here, first
        const float b1v = a.b.y1[l], b1h = a.b.y1[N + l], b2v = a.b.y2[l], b2h = a.b.y2[N + l];
        float gv1, gh1, gv2, gh2;
        LTop<IN>(a.aw1, d, l, i, j, gv1, gh1);
        LTop<IN>(a.aw2, d, l, i, j, gv2, gh2);
        const bool up = b < d.n3 - 1;
        auto dsg = [&](int di, int dj) {           // (D_s G_bar)(b, i+di, j+dj)
            return up ? nb<IN>(a.gbar, d, l + d.plane, i, j, di, dj) - nb<IN>(a.gbar, d, l, i, j, di, dj) : 0.f;
        };
        const float dvg = dv<IN>(a.gbar, d, l, i), dhg = dh<IN>(a.gbar, d, l, j);
        const float dvds = (IN || i < d.n1 - 1) ? dsg(1, 0) - dsg(0, 0) : 0.f;
        const float dhds = (IN || j < d.n2 - 1) ? dsg(0, 1) - dsg(0, 0) : 0.f;
        a.b.y1[l] = b1v + (dvg + a.g_w1 * gv1);
        a.b.y1[N + l] = b1h + (dhg + a.g_w1 * gh1);
        a.b.y2[l] = b2v + (dvds + a.g_w2 * gv2);
        a.b.y2[N + l] = b2h + (dhds + a.g_w2 * gh2);
    });
}

__global__ void __launch_bounds__(256) k_axpy(float* y, const float* x, float a, long long n) {
    for (long long l = blockIdx.x * 256ll + threadIdx.x; l < n; l += (long long)gridDim.x * 256)
        y[l] += a * x[l];
}

// Launch facts of one device: SM count and resident blocks of each kernel.
struct AdjInfo {
    int sms = 0;
    int res[5] = {0, 0, 0, 0, 0};
};

int resident_of(const void* fn) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, NTA, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return std::max(1, nb);
}

// Filled on the first launch with each device current (ordinals below 64;
// concurrent first launches write the same values).
const AdjInfo& adj_info();

// blocks of 32 x 8 threads: columns in x, persistent over the rows in y
dim3 adj_grid(const Dims& d, int resident, int sms) {
    const int gx = (d.n2 + BX - 1) / BX;
    const long long rb = ((long long)d.rows + BY - 1) / BY;
    const long long want = std::max(1ll, (long long)sms * std::max(1, resident) / gx);
    return dim3(gx, (unsigned)std::min({rb, want, 65535ll}));
}

// Resident blocks of each kernel and the SM count, filled once per device
// (std::call_once: concurrent first calls from several host threads wait for
// the one that fills it).
const AdjInfo& adj_info() {
    constexpr int kMaxDev = 64;
    static AdjInfo info[kMaxDev + 1];          // the last entry: device query failed
    static std::once_flag once[kMaxDev + 1];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
        cudaGetLastError();
        dev = kMaxDev;
    }
    AdjInfo& a = info[dev];
    std::call_once(once[dev], [&a] {
        a.res[0] = resident_of((const void*)k_adj_sums);
        a.res[1] = resident_of((const void*)k_adj_cube);
        a.res[2] = resident_of((const void*)k_adj_aux);
        a.res[3] = resident_of((const void*)k_adj_fin1);
        a.res[4] = resident_of((const void*)k_adj_fin2);
        a.sms = device_sms();
    });
    return a;
}

}  // namespace

int launch_axpy(float* y, const float* x, float a, long long n, cudaStream_t st) {
    if (n <= 0) return 0;
    const int grid = (int)std::min((n + 255) / 256, device_sms() * 8ll);
    k_axpy<<<grid, 256, 0, st>>>(y, x, a, n);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

size_t adjoint_workspace_bytes(long long n) {
    return (size_t)adj_stride(n) * 15 * sizeof(float) + 16 * sizeof(double);
}

int launch_adjoint_step(int n1, int n2, int n3, const float* const x[9], const float* const x1[9],
                        const float* const b1[9], float* const bo[9], const float* v, int v_pitch,
                        float* vbar, double* pbar, void* work, const double prm[16], cudaStream_t st) {
    const AdjInfo& info = adj_info();
    const int* res = info.res;
    AdjArgs a;
    a.d.n1 = n1; a.d.n2 = n2; a.d.n3 = n3; a.d.vp = v_pitch;
    a.d.rows = n3 * n1;
    a.d.plane = (long long)n1 * n2;
    a.d.N = (long long)n1 * n2 * n3;
    const long long N = a.d.N;
    a.x = SV{x[0], x[1], x[2], x[3], x[4], x[5], x[6], x[7], x[8]};
    a.x1 = SV{x1[0], x1[1], x1[2], x1[3], x1[4], x1[5], x1[6], x1[7], x1[8]};
    a.b1 = SV{b1[0], b1[1], b1[2], b1[3], b1[4], b1[5], b1[6], b1[7], b1[8]};
    a.b = SW{bo[0], bo[1], bo[2], bo[3], bo[4], bo[5], bo[6], bo[7], bo[8]};
    a.inplace = 1;
    for (int k = 0; k < 9; ++k)
        if (b1[k] != bo[k]) a.inplace = 0;
    a.v = v;
    a.vbar = vbar;
    a.pbar = pbar;
    // each region on a 256-byte boundary (the sums are doubles); the six
    // planes of aw1, aw2 keep the cube stride N inside their regions
    float* f = (float*)work;
    const long long P = adj_stride(N);
    a.gbar = f; a.aw1 = f + P; a.aw2 = f + 7 * P; a.s1b = f + 13 * P; a.t1b = f + 14 * P;
    a.sc = (double*)(f + 15 * P);
    a.g_u = (float)prm[0]; a.g_w1 = (float)prm[1]; a.g_w2 = (float)prm[2]; a.g_s = (float)prm[3];
    a.g_t = (float)prm[4]; a.g1 = (float)prm[5]; a.g2 = (float)prm[6]; a.g3 = (float)prm[7];
    a.g4 = (float)prm[8]; a.th1 = (float)prm[9]; a.th2 = (float)prm[10];
    a.mu_lo = (float)prm[11]; a.mu_hi = (float)prm[12];
    a.eps = prm[13]; a.alpha = prm[14]; a.beta = prm[15];
    a.g4d = prm[8]; a.g_w1d = prm[1];
    if (N == 0) return 0;
    if (cudaMemsetAsync(a.sc, 0, NSCAL * sizeof(double), st) != cudaSuccess) return -3;
    const dim3 blk(BX, BY);
    k_adj_sums<<<adj_grid(a.d, res[0], info.sms), blk, 0, st>>>(a);
    k_adj_cube<<<adj_grid(a.d, res[1], info.sms), blk, 0, st>>>(a);
    k_adj_aux<<<adj_grid(a.d, res[2], info.sms), blk, 0, st>>>(a);
    k_adj_fin1<<<adj_grid(a.d, res[3], info.sms), blk, 0, st>>>(a);
    k_adj_fin2<<<adj_grid(a.d, res[4], info.sms), blk, 0, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace gsstv
