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
// column; L^T is its exact transpose.  Four launches, a few device scalars
// for the global sums; nothing synchronises the host.
#include <cuda_runtime.h>

#include <algorithm>

#include "gsstv_internal.cuh"

namespace gsstv {
namespace {

constexpr int NTA = 256;

struct Dims {
    int n1, n2, n3;
    int vp;                                       // row pitch of v (floats)
    long long N;                                  // voxels
    __device__ __forceinline__ long long at(int b, int i, int j) const {
        return ((long long)b * n1 + i) * n2 + j;
    }
};

// the state views of one pass
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
    SW b;                         // adjoint of state k (written)
    const float* v;
    float* vbar;                  // += adjoint of v
    double* pbar;                 // += adjoints of eps, alpha, beta, omega
    double* sc;                   // NSCAL scalars, zeroed before the pass
    float *gbar, *aw1, *aw2, *s1b, *t1b, *atb;   // temporaries (N, 6N, 6N, N, N, N)
    double g_u, g_w1, g_w2, g_s, g_t, g1, g2, g3, g4, th1, th2, mu_lo, mu_hi, eps, alpha, beta;
};

// ---- stencils on dense cubes (value at (b, i, j) of an operator's output) ----
__device__ __forceinline__ float ld(const float* p, const Dims& d, int b, int i, int j) {
    return (i >= 0 && i < d.n1 && j >= 0 && j < d.n2 && b >= 0 && b < d.n3) ? p[d.at(b, i, j)] : 0.f;
}
// D_v x, D_h x, D_s x at (b, i, j)
__device__ __forceinline__ float dv(const float* x, const Dims& d, int b, int i, int j) {
    return i < d.n1 - 1 ? x[d.at(b, i + 1, j)] - x[d.at(b, i, j)] : 0.f;
}
__device__ __forceinline__ float dh(const float* x, const Dims& d, int b, int i, int j) {
    return j < d.n2 - 1 ? x[d.at(b, i, j + 1)] - x[d.at(b, i, j)] : 0.f;
}
// transposes: (D_v^T y)(i) = y(i-1) [i >= 1] - y(i) [i <= N1-2]
__device__ __forceinline__ float dvT(const float* y, const Dims& d, int b, int i, int j) {
    float r = 0.f;
    if (i >= 1) r += y[d.at(b, i - 1, j)];
    if (i <= d.n1 - 2) r -= y[d.at(b, i, j)];
    return r;
}
__device__ __forceinline__ float dhT(const float* y, const Dims& d, int b, int i, int j) {
    float r = 0.f;
    if (j >= 1) r += y[d.at(b, i, j - 1)];
    if (j <= d.n2 - 2) r -= y[d.at(b, i, j)];
    return r;
}
// D^T y for a dual pair y (2 planes of N)
__device__ __forceinline__ float dT(const float* y, const Dims& d, int b, int i, int j) {
    return dvT(y, d, b, i, j) + dhT(y + d.N, d, b, i, j);
}
// (D_s^T D^T y)(b) = (D^T y)(b-1) [b >= 1] - (D^T y)(b) [b <= N3-2]
__device__ __forceinline__ float dsT_dT(const float* y, const Dims& d, int b, int i, int j) {
    float r = 0.f;
    if (b >= 1) r += dT(y, d, b - 1, i, j);
    if (b <= d.n3 - 2) r -= dT(y, d, b, i, j);
    return r;
}
// masked dual-pair entries read by L
__device__ __forceinline__ float yvm(const float* y, const Dims& d, int b, int i, int j) {
    return (i >= 0 && i < d.n1 - 1 && j >= 0 && j < d.n2) ? y[d.at(b, i, j)] : 0.f;
}
__device__ __forceinline__ float yhm(const float* y, const Dims& d, int b, int i, int j) {
    return (i >= 0 && i < d.n1 && j >= 0 && j < d.n2 - 1) ? y[d.N + d.at(b, i, j)] : 0.f;
}
// L y at (b, i, j): out[k], k = 2 g + c (g grid, c = vertical / horizontal)
__device__ __forceinline__ void Lop(const float* y, const Dims& d, int b, int i, int j, float out[6]) {
    const float v00 = yvm(y, d, b, i, j), vm0 = yvm(y, d, b, i - 1, j), v01 = yvm(y, d, b, i, j + 1),
                vm1 = yvm(y, d, b, i - 1, j + 1);
    const float h00 = yhm(y, d, b, i, j), h0m = yhm(y, d, b, i, j - 1), h10 = yhm(y, d, b, i + 1, j),
                h1m = yhm(y, d, b, i + 1, j - 1);
    const bool mv = i < d.n1 - 1, mh = j < d.n2 - 1;
    out[0] = mv ? v00 : 0.f;
    out[1] = mv ? 0.25f * (h00 + h0m + h10 + h1m) : 0.f;
    out[2] = mh ? 0.25f * (v00 + vm0 + v01 + vm1) : 0.f;
    out[3] = mh ? h00 : 0.f;
    out[4] = 0.5f * (v00 + vm0);
    out[5] = 0.5f * (h00 + h0m);
}
// component k of w at (b, i, j), zero outside the image and where L's
// output is structurally zero (grid 0 on the last row, grid 1 on the last column)
__device__ __forceinline__ float wk(const float* w, const Dims& d, int k, int b, int i, int j) {
    if (i < 0 || i >= d.n1 || j < 0 || j >= d.n2) return 0.f;
    if (k < 2 && i == d.n1 - 1) return 0.f;
    if ((k == 2 || k == 3) && j == d.n2 - 1) return 0.f;
    return w[(long long)k * d.N + d.at(b, i, j)];
}
// L^T w at (b, i, j): (vertical, horizontal)
__device__ __forceinline__ void LTop(const float* w, const Dims& d, int b, int i, int j, float& gv, float& gh) {
    const bool mv = i < d.n1 - 1, mh = j < d.n2 - 1;
    gv = mv ? (wk(w, d, 0, b, i, j) +
               0.25f * (wk(w, d, 2, b, i, j) + wk(w, d, 2, b, i + 1, j) + wk(w, d, 2, b, i, j - 1) +
                        wk(w, d, 2, b, i + 1, j - 1)) +
               0.5f * (wk(w, d, 4, b, i, j) + wk(w, d, 4, b, i + 1, j)))
            : 0.f;
    gh = mh ? (0.25f * (wk(w, d, 1, b, i, j) + wk(w, d, 1, b, i, j + 1) + wk(w, d, 1, b, i - 1, j) +
                        wk(w, d, 1, b, i - 1, j + 1)) +
               wk(w, d, 3, b, i, j) + 0.5f * (wk(w, d, 5, b, i, j) + wk(w, d, 5, b, i, j + 1)))
            : 0.f;
}

__device__ __forceinline__ void coords(const Dims& d, long long l, int& b, int& i, int& j) {
    j = (int)(l % d.n2);
    const long long r = l / d.n2;
    i = (int)(r % d.n1);
    b = (int)(r / d.n1);
}

__device__ __forceinline__ double block_sum_d(double x, double* buf) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) buf[w] = x;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += buf[k];
    return r;                                      // valid on thread 0
}

// q = y4 + g4 (u' + s' + t') - g4 v at voxel l = (b, i, j)
__device__ __forceinline__ float q_at(const AdjArgs& a, long long l, int b, int i, int j) {
    const float up = 2.f * a.x1.u[l] - a.x.u[l], sp = 2.f * a.x1.s[l] - a.x.s[l], tp = 2.f * a.x1.t[l] - a.x.t[l];
    const float v = a.v[((long long)b * a.d.n1 + i) * a.d.vp + j];
    return a.x.y4[l] + (float)a.g4 * (up + sp + tp) - (float)a.g4 * v;
}

// R0: |q|^2, q . y4_bar+, |a_s|_1, |a_t|_1
__global__ void __launch_bounds__(NTA) k_adj_r0(const AdjArgs a) {
    __shared__ double buf[NTA / 32];
    double qq = 0, qb = 0, l1s = 0, l1t = 0;
    for (long long l = blockIdx.x * (long long)NTA + threadIdx.x; l < a.d.N; l += (long long)gridDim.x * NTA) {
        int b, i, j;
        coords(a.d, l, b, i, j);
        const double q = q_at(a, l, b, i, j);
        qq += q * q;
        qb += q * a.b1.y4[l];
        l1s += fabs((double)a.x.s[l] - a.g_s * a.x.y4[l]);
        const float at = a.x.t[l] - (float)a.g_t * (dvT(a.x.y3, a.d, b, i, j) + a.x.y4[l]);
        l1t += fabs((double)at);
    }
    const double r0 = block_sum_d(qq, buf), r1 = block_sum_d(qb, buf), r2 = block_sum_d(l1s, buf),
                 r3 = block_sum_d(l1t, buf);
    if (threadIdx.x == 0) {
        atomicAdd(a.sc + QQ, r0);
        atomicAdd(a.sc + QB, r1);
        atomicAdd(a.sc + L1S, r2);
        atomicAdd(a.sc + L1T, r3);
    }
}

// R1: l2 step, dual-ascent transposes, extrapolation, box and group shrink;
// sums for the l1 adjoints and the omega adjoint
__global__ void __launch_bounds__(NTA) k_adj_r1(const AdjArgs a) {
    __shared__ double buf[NTA / 32];
    const Dims& d = a.d;
    const long long N = d.N;
    const double nq = sqrt(a.sc[QQ]);
    const bool l2act = nq > a.eps * a.g4;
    const double qdot = l2act ? a.sc[QB] / nq : 0.0;           // q^ . y4_bar+
    const float fk = l2act ? (float)(a.eps * a.g4 / nq) : 0.f;
    const float qh_scale = l2act ? (float)(1.0 / nq) : 0.f;
    double ss = 0, ns = 0, st = 0, nt = 0, th = 0;
    for (long long l = blockIdx.x * (long long)NTA + threadIdx.x; l < N; l += (long long)gridDim.x * NTA) {
        int b, i, j;
        coords(d, l, b, i, j);
        // y4+ = (1 - c) q
        const float y4b = a.b1.y4[l];
        const float qbar = l2act ? y4b - fk * (y4b - q_at(a, l, b, i, j) * qh_scale * (float)qdot) : 0.f;
        a.vbar[l] += -(float)a.g4 * qbar;
        // adjoints of the extrapolated primals
        const float ub_ = (float)a.g4 * qbar + (float)a.g2 * dsT_dT(a.b1.y2, d, b, i, j) +
                          (float)a.g1 * dT(a.b1.y1, d, b, i, j);
        const float sb_ = (float)a.g4 * qbar;
        const float tb_ = (float)a.g4 * qbar + (float)a.g3 * dvT(a.b1.y3, d, b, i, j);
        float l1w[6], l2w[6];
        Lop(a.b1.y1, d, b, i, j, l1w);
        Lop(a.b1.y2, d, b, i, j, l2w);
        // u+ = box(a_u): the adjoint passes where mu_lo < u+ < mu_hi
        const float u1 = a.x1.u[l];
        const float u1bar = a.b1.u[l] + 2.f * ub_;
        const float aub = (u1 > (float)a.mu_lo && u1 < (float)a.mu_hi) ? u1bar : 0.f;
        a.b.u[l] = -ub_ + aub;
        a.gbar[l] = -(float)a.g_u * aub;
        // s, t: totals for the projections (finished in R2)
        const float s1bar = a.b1.s[l] + 2.f * sb_, t1bar = a.b1.t[l] + 2.f * tb_;
        a.s1b[l] = s1bar;
        a.t1b[l] = t1bar;
        a.b.s[l] = -sb_;
        a.b.t[l] = -tb_;
        const float s1 = a.x1.s[l], t1 = a.x1.t[l];
        if (s1 != 0.f) { ss += (s1 > 0.f ? s1bar : -s1bar); ns += 1.0; }
        if (t1 != 0.f) { st += (t1 > 0.f ? t1bar : -t1bar); nt += 1.0; }
        // duals keep their own adjoint; y4 gets q_bar (more in R2)
        a.b.y1[l] = a.b1.y1[l];
        a.b.y1[N + l] = a.b1.y1[N + l];
        a.b.y2[l] = a.b1.y2[l];
        a.b.y2[N + l] = a.b1.y2[N + l];
        a.b.y3[l] = a.b1.y3[l];
        a.b.y4[l] = qbar;
        // w: a_w = w + g L y, group shrink with threshold th
        float ly1[6], ly2[6];
        Lop(a.x.y1, d, b, i, j, ly1);
        Lop(a.x.y2, d, b, i, j, ly2);
#pragma unroll
        for (int set = 0; set < 2; ++set) {
            const float* w = set ? a.x.w2 : a.x.w1;
            const float* wb1 = set ? a.b1.w2 : a.b1.w1;
            const float* lw = set ? l2w : l1w;
            const float* ly = set ? ly2 : ly1;
            float* bw = set ? a.b.w2 : a.b.w1;
            float* aw = set ? a.aw2 : a.aw1;
            const float gw = (float)(set ? a.g_w2 : a.g_w1);
            const float gy = (float)(set ? a.g2 : a.g1);
            const float thr = (float)(set ? a.th2 : a.th1);
#pragma unroll
            for (int g = 0; g < 3; ++g) {
                const long long kv = (long long)(2 * g) * N + l, kh = (long long)(2 * g + 1) * N + l;
                const float xv = w[kv] + gw * ly[2 * g], xh = w[kh] + gw * ly[2 * g + 1];
                const float wbv = -gy * lw[2 * g], wbh = -gy * lw[2 * g + 1];     // adjoint of w'
                const float pv = wb1[kv] + 2.f * wbv, ph = wb1[kh] + 2.f * wbh;   // total of w+
                const float n = sqrtf(xv * xv + xh * xh);
                float av = 0.f, ah = 0.f;
                if (n > thr) {
                    const float xhv = xv / n, xhh = xh / n;
                    const float dot = xhv * pv + xhh * ph;
                    const float k1 = 1.f - thr / n, k2 = thr / n;
                    av = k1 * pv + k2 * xhv * dot;
                    ah = k1 * ph + k2 * xhh * dot;
                    if (set == 0) th += -(double)dot;
                }
                aw[kv] = av;
                aw[kh] = ah;
                bw[kv] = -wbv + av;
                bw[kh] = -wbh + ah;
            }
        }
    }
    const double r0 = block_sum_d(ss, buf), r1 = block_sum_d(ns, buf), r2 = block_sum_d(st, buf),
                 r3 = block_sum_d(nt, buf), r4 = block_sum_d(th, buf);
    if (threadIdx.x == 0) {
        atomicAdd(a.sc + SS, r0);
        atomicAdd(a.sc + NS, r1);
        atomicAdd(a.sc + ST, r2);
        atomicAdd(a.sc + NT_, r3);
        atomicAdd(a.sc + TH1, r4);
        if (blockIdx.x == 0 && l2act) atomicAdd(a.pbar + 0, -a.g4 * qdot);
    }
}

// R2: l1 adjoints, y4 and the stencils of G_bar and the group-shrink adjoints
// onto y1, y2
__global__ void __launch_bounds__(NTA) k_adj_r2(const AdjArgs a) {
    const Dims& d = a.d;
    const long long N = d.N;
    const bool in_s = a.sc[L1S] <= a.alpha, in_t = a.sc[L1T] <= a.beta;
    const float ks = (!in_s && a.sc[NS] > 0) ? (float)(a.sc[SS] / a.sc[NS]) : 0.f;
    const float kt = (!in_t && a.sc[NT_] > 0) ? (float)(a.sc[ST] / a.sc[NT_]) : 0.f;
    for (long long l = blockIdx.x * (long long)NTA + threadIdx.x; l < N; l += (long long)gridDim.x * NTA) {
        int b, i, j;
        coords(d, l, b, i, j);
        const float s1 = a.x1.s[l], t1 = a.x1.t[l];
        const float asb = in_s ? a.s1b[l] : (s1 != 0.f ? a.s1b[l] - (s1 > 0.f ? ks : -ks) : 0.f);
        const float atb = in_t ? a.t1b[l] : (t1 != 0.f ? a.t1b[l] - (t1 > 0.f ? kt : -kt) : 0.f);
        a.b.s[l] += asb;
        a.b.t[l] += atb;
        a.atb[l] = atb;
        a.b.y4[l] += a.gbar[l] - (float)a.g_s * asb - (float)a.g_t * atb;
        // y1 += D G_bar + g_w1 L^T aw1;  y2 += D D_s G_bar + g_w2 L^T aw2
        float gv1, gh1, gv2, gh2;
        LTop(a.aw1, d, b, i, j, gv1, gh1);
        LTop(a.aw2, d, b, i, j, gv2, gh2);
        const float dsg_here = b < d.n3 - 1 ? 1.f : 0.f;
        // D_s G at (b, i, j) and its neighbours for D (D_s G)
        auto dsg = [&](int ii, int jj) {
            return dsg_here != 0.f ? ld(a.gbar, d, b + 1, ii, jj) - ld(a.gbar, d, b, ii, jj) : 0.f;
        };
        a.b.y1[l] += dv(a.gbar, d, b, i, j) + (float)a.g_w1 * gv1;
        a.b.y1[N + l] += dh(a.gbar, d, b, i, j) + (float)a.g_w1 * gh1;
        const float dvds = i < d.n1 - 1 ? dsg(i + 1, j) - dsg(i, j) : 0.f;
        const float dhds = j < d.n2 - 1 ? dsg(i, j + 1) - dsg(i, j) : 0.f;
        a.b.y2[l] += dvds + (float)a.g_w2 * gv2;
        a.b.y2[N + l] += dhds + (float)a.g_w2 * gh2;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (!in_s) atomicAdd(a.pbar + 1, (double)ks);
        if (!in_t) atomicAdd(a.pbar + 2, (double)kt);
        atomicAdd(a.pbar + 3, a.g_w1 * a.sc[TH1]);
    }
}

// R3: y3 += -g_t D_v a_t_bar
__global__ void __launch_bounds__(NTA) k_adj_r3(const AdjArgs a) {
    for (long long l = blockIdx.x * (long long)NTA + threadIdx.x; l < a.d.N; l += (long long)gridDim.x * NTA) {
        int b, i, j;
        coords(a.d, l, b, i, j);
        a.b.y3[l] += -(float)a.g_t * dv(a.atb, a.d, b, i, j);
    }
}

__global__ void __launch_bounds__(NTA) k_axpy(float* y, const float* x, float a, long long n) {
    for (long long l = blockIdx.x * (long long)NTA + threadIdx.x; l < n; l += (long long)gridDim.x * NTA)
        y[l] += a * x[l];
}

}  // namespace

int launch_axpy(float* y, const float* x, float a, long long n, cudaStream_t st) {
    if (n <= 0) return 0;
    const int grid = (int)std::min((n + NTA - 1) / NTA, 152ll * 8);
    k_axpy<<<grid, NTA, 0, st>>>(y, x, a, n);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

size_t adjoint_workspace_bytes(long long n) {
    return (size_t)n * 16 * sizeof(float) + 16 * sizeof(double);
}

int launch_adjoint_step(int n1, int n2, int n3, const float* const x[9], const float* const x1[9],
                        const float* const b1[9], float* const bo[9], const float* v, int v_pitch,
                        float* vbar, double* pbar, void* work, const double prm[16], cudaStream_t st) {
    AdjArgs a;
    a.d.n1 = n1; a.d.n2 = n2; a.d.n3 = n3; a.d.vp = v_pitch;
    a.d.N = (long long)n1 * n2 * n3;
    const long long N = a.d.N;
    a.x = SV{x[0], x[1], x[2], x[3], x[4], x[5], x[6], x[7], x[8]};
    a.x1 = SV{x1[0], x1[1], x1[2], x1[3], x1[4], x1[5], x1[6], x1[7], x1[8]};
    a.b1 = SV{b1[0], b1[1], b1[2], b1[3], b1[4], b1[5], b1[6], b1[7], b1[8]};
    a.b = SW{bo[0], bo[1], bo[2], bo[3], bo[4], bo[5], bo[6], bo[7], bo[8]};
    a.v = v;
    a.vbar = vbar;
    a.pbar = pbar;
    float* f = (float*)work;
    a.gbar = f; a.aw1 = f + N; a.aw2 = f + 7 * N; a.s1b = f + 13 * N; a.t1b = f + 14 * N; a.atb = f + 15 * N;
    a.sc = (double*)(f + 16 * N);
    a.g_u = prm[0]; a.g_w1 = prm[1]; a.g_w2 = prm[2]; a.g_s = prm[3]; a.g_t = prm[4];
    a.g1 = prm[5]; a.g2 = prm[6]; a.g3 = prm[7]; a.g4 = prm[8];
    a.th1 = prm[9]; a.th2 = prm[10]; a.mu_lo = prm[11]; a.mu_hi = prm[12];
    a.eps = prm[13]; a.alpha = prm[14]; a.beta = prm[15];
    if (cudaMemsetAsync(a.sc, 0, NSCAL * sizeof(double), st) != cudaSuccess) return -3;
    const int grid = (int)std::max(1ll, std::min((N + NTA - 1) / NTA, 152ll * 8));
    k_adj_r0<<<grid, NTA, 0, st>>>(a);
    k_adj_r1<<<grid, NTA, 0, st>>>(a);
    k_adj_r2<<<grid, NTA, 0, st>>>(a);
    k_adj_r3<<<grid, NTA, 0, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace gsstv
