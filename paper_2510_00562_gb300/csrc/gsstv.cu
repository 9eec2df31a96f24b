// Host driver and C ABI of libgsstv (declared in include/gsstv.h).
//
// One iteration of Algorithm 1 is nine launches on the handle's stream:
//   K1  fused stencil pass (u, w1, w2, y1, y2 and the l1 window statistics);
//   W, F  one retry window for a threshold whose K1 window missed, and its
//       finish (one CTA);
//   R0, R1, R2  radix passes of the exact l1-threshold search (each returns at
//       once unless the previous step left that level pending);
//   G, F  gather of the bracket bin and its finish (same early return);
//   K2  light pass (s, t, y3, y4 and the l2-ball norm).
// Every scalar that couples the iteration (the thresholds tau_s, tau_t and the
// l2-ball scale c) stays on the device, so a block of iterations can be
// captured once into a CUDA graph and replayed; the host synchronises only
// for the stopping rule (Eq. 28) and for the final error check.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

#include "gsstv.h"
#include "gsstv_internal.cuh"

using namespace gsstv;

struct gsstv_handle {
    Geom g{};
    gsstv_params p{};
    cudaStream_t st = nullptr;
    cudaStream_t cap = nullptr;   // private stream used only to capture graphs
    cudaStream_t cap2 = nullptr;  // and one for the bodies of conditional graph nodes
    int esz = 4;
    void *u[2]{}, *s[2]{}, *t[2]{}, *y3[2]{}, *q[2]{};
    void *w1[2]{}, *w2[2]{}, *y1[2]{}, *y2[2]{};
    float* v = nullptr;
    float* tmp = nullptr;         // dense float32 scratch for host copies (16-bit storage)
    void* adj_work = nullptr;     // scratch of gsstv_vjp_step (allocated on first use)
    Scal* sc = nullptr;
    L1Work l1{};
    double* k2_part = nullptr;
    int k2_cap = 0;
    int k1_ctas = 0;
    int parity = 0;               // ping-pong index that holds the current state
    int k1_variant = 1;           // 1: TMA-fed K1, 0: cooperative-load K1 (GSSTV_K1=coop)
    int k1_chunk = 0;             // bands per K1 CTA (0: the wave/prologue model's choice)
    K1Maps maps[2];               // tensor maps of the buffers read at parity 0 / 1
    cudaGraphExec_t gexec[2]{};
    int graph_len = 0;
    int timing = 0;
    std::vector<cudaEvent_t> ev;
    int ev_used = 0;
    // graphs with K1 between timing events: one per parity and slot of 2 x len
    // events of the pool (kept, like the untimed graphs, until the launch
    // shape changes)
    static constexpr int kTimedSlots = 16;
    cudaGraphExec_t timed_exec[2][kTimedSlots]{};
    int timed_len = 0;
    gsstv_stats stats{};
    int64_t bytes = 0;
    std::vector<void*> allocs;
};

namespace {

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? GSSTV_OK : GSSTV_ERR_CUDA; }
#define TRY(x) do { int rc__ = (x); if (rc__ != GSSTV_OK) return rc__; } while (0)

bool finite_nonneg(double x) { return std::isfinite(x) && x >= 0.0; }
bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

int check_params(const gsstv_params* p) {
    if (!p) return GSSTV_ERR_ARG;
    if (!finite_nonneg(p->eps) || !finite_nonneg(p->alpha) || !finite_nonneg(p->beta) || !finite_nonneg(p->omega))
        return GSSTV_ERR_ARG;
    if (!std::isfinite(p->mu_lo) || !std::isfinite(p->mu_hi) || !(p->mu_lo < p->mu_hi)) return GSSTV_ERR_ARG;
    const double gam[] = {p->gamma_u, p->gamma_w1, p->gamma_w2, p->gamma_s, p->gamma_t,
                          p->gamma_y1, p->gamma_y2, p->gamma_y3, p->gamma_y4};
    for (double x : gam)
        if (!finite_pos(x)) return GSSTV_ERR_ARG;
    if (p->max_iter < 0 || p->check_every < 1 || p->graph_iters < 0) return GSSTV_ERR_ARG;
    if (!(p->tol >= 0.0) || !std::isfinite(p->tol)) return GSSTV_ERR_ARG;
    if (p->storage < GSSTV_FP32 || p->storage > GSSTV_FP16) return GSSTV_ERR_ARG;
    if (p->tau_mode != GSSTV_TAU_AUTO && p->tau_mode != GSSTV_TAU_EXACT) return GSSTV_ERR_ARG;
    return GSSTV_OK;
}

int dalloc(gsstv_handle* h, void** out, size_t bytes) {
    *out = nullptr;
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(out, bytes) != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        return GSSTV_ERR_OOM;
    }
    h->allocs.push_back(*out);
    h->bytes += (int64_t)bytes;
    if (cudaMemsetAsync(*out, 0, bytes, h->st) != cudaSuccess) return GSSTV_ERR_CUDA;
    return GSSTV_OK;
}

void free_all(gsstv_handle* h) {
    for (int k = 0; k < 2; ++k)
        if (h->gexec[k]) { cudaGraphExecDestroy(h->gexec[k]); h->gexec[k] = nullptr; }
    cudaStreamSynchronize(h->st);
    for (auto& row : h->timed_exec)
        for (cudaGraphExec_t& x : row)
            if (x) { cudaGraphExecDestroy(x); x = nullptr; }
    for (cudaEvent_t e : h->ev) if (e) cudaEventDestroy(e);
    h->ev.clear();
    if (h->cap) { cudaStreamDestroy(h->cap); h->cap = nullptr; }
    if (h->cap2) { cudaStreamDestroy(h->cap2); h->cap2 = nullptr; }
    for (void* p : h->allocs) cudaFree(p);
    h->allocs.clear();
}

void destroy_graphs(gsstv_handle* h) {
    for (int k = 0; k < 2; ++k)
        if (h->gexec[k]) { cudaGraphExecDestroy(h->gexec[k]); h->gexec[k] = nullptr; }
    h->graph_len = 0;
    if (h->timed_len) cudaStreamSynchronize(h->st);
    for (auto& row : h->timed_exec)
        for (cudaGraphExec_t& x : row)
            if (x) { cudaGraphExecDestroy(x); x = nullptr; }
    h->timed_len = 0;
}

IterBufs bufs(const gsstv_handle* h, int par) {
    const int n = par ^ 1;
    IterBufs b;
    b.u = h->u[par]; b.s = h->s[par]; b.t = h->t[par]; b.y3 = h->y3[par]; b.q = h->q[par];
    b.w1 = h->w1[par]; b.w2 = h->w2[par]; b.y1 = h->y1[par]; b.y2 = h->y2[par];
    b.u_n = h->u[n]; b.s_n = h->s[n]; b.t_n = h->t[n]; b.y3_n = h->y3[n]; b.q_n = h->q[n];
    b.w1_n = h->w1[n]; b.w2_n = h->w2[n]; b.y1_n = h->y1[n]; b.y2_n = h->y2[n];
    b.v = h->v;
    return b;
}

IterParams iparams(const gsstv_handle* h, int par) {
    const gsstv_params& p = h->p;
    IterParams ip;
    ip.gamma_u = (float)p.gamma_u; ip.gamma_w1 = (float)p.gamma_w1; ip.gamma_w2 = (float)p.gamma_w2;
    ip.gamma_s = (float)p.gamma_s; ip.gamma_t = (float)p.gamma_t;
    ip.gamma_y1 = (float)p.gamma_y1; ip.gamma_y2 = (float)p.gamma_y2;
    ip.gamma_y3 = (float)p.gamma_y3; ip.gamma_y4 = (float)p.gamma_y4;
    ip.thr_w1 = (float)(p.gamma_w1 * p.omega);
    ip.thr_w2 = (float)p.gamma_w2;
    ip.mu_lo = (float)p.mu_lo; ip.mu_hi = (float)p.mu_hi;
    ip.eps = p.eps;
    ip.parity = par;
    ip.tau_exact = p.tau_mode == GSSTV_TAU_EXACT;
    ip.max_iter = 0;                   // the stopping rule runs on the host for a single handle
    ip.check_every = 0;
    ip.tol = 0.0;
    ip.live = nullptr;
    return ip;
}

int map_launch(int rc) { return rc == 0 ? GSSTV_OK : rc == -1 ? GSSTV_ERR_ARG : GSSTV_ERR_CUDA; }

// While `st` is being captured into a graph: the launches that body(stream)
// enqueues become the body of a conditional node, run only when the launch
// that decide(cond) enqueues just before it (K1's window finish, or a gate
// kernel) sets the condition: after K1's window finish most passes need no
// threshold search, and the seven search launches would each start and
// return at once.  The body is captured from the side stream `side`.
template <typename D, typename F>
int capture_if_search(cudaStream_t st, cudaStream_t side, D&& decide, F&& body) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    TRY(cuda_rc(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd)));
    if (cs != cudaStreamCaptureStatusActive) return GSSTV_ERR_INTERNAL;
    cudaGraphConditionalHandle cond = 0;
    TRY(cuda_rc(cudaGraphConditionalHandleCreate(&cond, g, 0, cudaGraphCondAssignDefault)));
    TRY(decide(cond));
    TRY(cuda_rc(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd)));
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeIf;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    TRY(cuda_rc(cudaGraphAddNode(&node, g, deps, nullptr, nd, &np)));
    TRY(cuda_rc(cudaStreamBeginCaptureToGraph(side, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal)));
    const int rc = body(side);
    cudaGraph_t body_graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(side, &body_graph);
    TRY(rc);
    TRY(cuda_rc(e));
    TRY(cuda_rc(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies)));
    return GSSTV_OK;
}

// One iteration from parity `par` (reads buffers par, writes par ^ 1) on `st`;
// in_graph: `st` is being captured (the search launches then sit behind a
// conditional node).
int enqueue_iteration(gsstv_handle* h, int par, bool timed, cudaStream_t st, bool in_graph = false) {
    const IterBufs b = bufs(h, par);
    const IterParams ip = iparams(h, par);
    const int sto = h->p.storage;
    if (timed) {
        if (h->ev_used + 2 > (int)h->ev.size()) return GSSTV_ERR_INTERNAL;
        // inside a capture only an external record becomes a graph node
        TRY(cuda_rc(in_graph ? cudaEventRecordWithFlags(h->ev[h->ev_used], st, cudaEventRecordExternal)
                             : cudaEventRecord(h->ev[h->ev_used], st)));
    }
    const SlabPart whole = whole_cube(h->g);
    if (h->k1_variant == 1)
        TRY(map_launch(launch_k1_tma(sto, h->g, h->maps[par], b, ip, h->sc, h->l1, h->k1_chunk, whole, st)));
    else
        TRY(map_launch(launch_k1(sto, h->g, b, ip, h->sc, h->l1, h->k1_ctas, st)));
    if (timed) {
        TRY(cuda_rc(in_graph ? cudaEventRecordWithFlags(h->ev[h->ev_used + 1], st, cudaEventRecordExternal)
                             : cudaEventRecord(h->ev[h->ev_used + 1], st)));
        h->ev_used += 2;
    }
    // the TMA-fed K1 leaves its window's finish to a launch of its own (the
    // cooperative K1 finishes it in its last CTA); in a graph that launch, or
    // a gate kernel, decides whether the search launches run
    auto k1_finish = [&](int gated, cudaGraphConditionalHandle cond) -> int {
        if (h->k1_variant == 1)
            return map_launch(launch_search_finish(2, h->sc, h->l1, 2, h->l1.k1_n, h->l1.k1_s,
                                                   k1_tma_grid(h->g, whole, h->k1_chunk), st, gated, cond));
        return gated ? map_launch(launch_search_gate(&h->sc, 1, cond, st)) : GSSTV_OK;
    };
    auto search = [&](cudaStream_t s) -> int {
        TRY(map_launch(launch_window(sto, h->g, b, ip, h->sc, h->l1, h->k1_ctas, whole, s)));
        TRY(map_launch(launch_search_finish(0, h->sc, h->l1, 2, h->l1.k1_n, h->l1.k1_s,
                                            window_grid(h->g, whole, h->k1_ctas), s)));
        for (int level = 0; level < 3; ++level)
            TRY(map_launch(launch_fallback(sto, level, h->g, b, ip, h->sc, h->l1, whole, s)));
        TRY(map_launch(launch_gather(sto, h->g, b, ip, h->sc, h->l1, whole, s)));
        TRY(map_launch(launch_search_finish(1, h->sc, h->l1, 2, nullptr, nullptr, 0, s)));
        return GSSTV_OK;
    };
    if (in_graph) {
        TRY(capture_if_search(st, h->cap2, [&](cudaGraphConditionalHandle c) { return k1_finish(1, c); }, search));
    } else {
        TRY(k1_finish(0, 0));
        TRY(search(st));
    }
    TRY(map_launch(launch_k2(sto, h->g, b, ip, h->sc, h->k2_part, h->k2_cap, whole, st)));
    return GSSTV_OK;
}

// Captures `len` iterations starting at parity `par` on the private capture
// stream (the caller's stream may be the legacy default stream, which cannot
// be captured); the executable graph is launched on the caller's stream.
// timed: each iteration's K1 between two of the handle's timing events (a
// graph built for one launch, since its events are read afterwards).
int build_graph_exec(gsstv_handle* h, int par, int len, bool timed, cudaGraphExec_t* out) {
    cudaGraph_t graph = nullptr;
    TRY(cuda_rc(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal)));
    int rc = GSSTV_OK;
    int p = par;
    for (int k = 0; k < len && rc == GSSTV_OK; ++k) {
        rc = enqueue_iteration(h, p, timed, h->cap, true);
        p ^= 1;
    }
    cudaError_t e = cudaStreamEndCapture(h->cap, &graph);
    if (rc != GSSTV_OK) { if (graph) cudaGraphDestroy(graph); return rc; }
    if (e != cudaSuccess) return GSSTV_ERR_CUDA;
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    return cuda_rc(e);
}
int build_graph(gsstv_handle* h, int par, int len) { return build_graph_exec(h, par, len, false, &h->gexec[par]); }

int flush_timing(gsstv_handle* h) {
    if (h->ev_used == 0) return GSSTV_OK;
    TRY(cuda_rc(cudaStreamSynchronize(h->st)));
    for (int k = 0; k + 1 < h->ev_used; k += 2) {
        float ms = 0.f;
        TRY(cuda_rc(cudaEventElapsedTime(&ms, h->ev[k], h->ev[k + 1])));
        h->stats.k1_ms += ms;
        h->stats.k1_launches++;
    }
    h->ev_used = 0;
    return GSSTV_OK;
}

// n iterations, no stopping test
int run_block(gsstv_handle* h, int n) {
    const int G = h->p.graph_iters > 0 ? ((h->p.graph_iters + 1) / 2) * 2 : 0;   // even: parity returns
    while (n > 0) {
        if (!h->timing && G > 0 && n >= G) {
            if (h->graph_len != G) destroy_graphs(h);
            if (!h->gexec[h->parity]) TRY(build_graph(h, h->parity, G));
            h->graph_len = G;
            TRY(cuda_rc(cudaGraphLaunch(h->gexec[h->parity], h->st)));
            n -= G;
            h->stats.iterations += G;
        } else if (h->timing && G > 0 && n >= G && 2 * G * gsstv_handle::kTimedSlots <= (int)h->ev.size()) {
            // the same graphs with K1 between timing events: the graph of
            // slot k records events [2 G k, 2 G (k + 1)) of the pool, which
            // are read (flush_timing) before the slot is launched again
            if (h->ev_used % (2 * G) != 0 || h->ev_used + 2 * G > 2 * G * gsstv_handle::kTimedSlots)
                TRY(flush_timing(h));
            if (h->timed_len != G) destroy_graphs(h);
            h->timed_len = G;
            cudaGraphExec_t& x = h->timed_exec[h->parity][h->ev_used / (2 * G)];
            if (!x) TRY(build_graph_exec(h, h->parity, G, true, &x));     // advances ev_used by 2 G
            else h->ev_used += 2 * G;
            TRY(cuda_rc(cudaGraphLaunch(x, h->st)));
            n -= G;
            h->stats.iterations += G;
        } else {
            if (h->timing && h->ev_used + 2 > (int)h->ev.size()) TRY(flush_timing(h));
            TRY(enqueue_iteration(h, h->parity, h->timing != 0, h->st));
            h->parity ^= 1;
            --n;
            h->stats.iterations += 1;
        }
    }
    return GSSTV_OK;
}

// Shapes a handle accepts: sides >= 1, N1, N2 <= 2^20, N3 <= 2^16, and six
// stacked cubes addressable with 32-bit offsets (the stencil kernel's w
// buffers).
bool shape_ok(int n1, int n2, int n3) {
    if (n1 < 1 || n2 < 1 || n3 < 1 || n1 > (1 << 20) || n2 > (1 << 20) || n3 > (1 << 16)) return false;
    const long long cube = (long long)n3 * n1 * (((long long)n2 + 7) / 8 * 8);
    return cube * 6 < (1ll << 32);
}

int read_scalars(gsstv_handle* h, Scal* out) {
    TRY(cuda_rc(cudaMemcpyAsync(out, h->sc, sizeof(Scal), cudaMemcpyDeviceToHost, h->st)));
    return cuda_rc(cudaStreamSynchronize(h->st));
}

int error_of(const Scal& s) {
    if (s.error & 1) return GSSTV_ERR_NONFINITE;
    if (s.error & 4) return GSSTV_ERR_TIMEOUT;
    if (s.error) return GSSTV_ERR_INTERNAL;
    return GSSTV_OK;
}

Scal initial_scalars(const gsstv_params& p) {
    Scal s;
    std::memset(&s, 0, sizeof(s));
    s.radius[0] = p.alpha;
    s.radius[1] = p.beta;
    for (int v = 0; v < 2; ++v) {
        s.ctl[v].window_ok = 1;       // first window (0, 0]: is the vector inside the ball?
        s.ctl[v].need = NEED_NONE;
    }
    return s;
}

int upload_scalars(gsstv_handle* h, const Scal& s) {
    Scal tmp = s;
    TRY(cuda_rc(cudaMemcpyAsync(h->sc, &tmp, sizeof(Scal), cudaMemcpyHostToDevice, h->st)));
    return cuda_rc(cudaStreamSynchronize(h->st));
}

}  // namespace

extern "C" {

void gsstv_default_params(gsstv_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->eps = 1.0; p->alpha = 1.0; p->beta = 1.0; p->omega = 0.03;
    p->mu_lo = 0.0; p->mu_hi = 1.0;
    p->gamma_u = 1.0 / 13.0; p->gamma_w1 = 0.25; p->gamma_w2 = 0.25;
    p->gamma_s = 1.0; p->gamma_t = 1.0 / 3.0;
    p->gamma_y1 = p->gamma_y2 = p->gamma_y3 = p->gamma_y4 = 0.2;
    p->max_iter = 1000; p->tol = 0.0; p->check_every = 100;
    p->storage = GSSTV_FP32; p->tau_mode = GSSTV_TAU_AUTO; p->graph_iters = 16;
}

int gsstv_create(gsstv_handle** out, int n1, int n2, int n3, const gsstv_params* p, void* stream) {
    if (!out) return GSSTV_ERR_ARG;
    *out = nullptr;
    if (!shape_ok(n1, n2, n3)) return GSSTV_ERR_ARG;
    TRY(check_params(p));
    gsstv_handle* h = new gsstv_handle();
    h->p = *p;
    h->st = (cudaStream_t)stream;
    h->esz = p->storage == GSSTV_FP32 ? 4 : 2;
    h->g.n1 = n1; h->g.n2 = n2; h->g.n3 = n3;
    h->g.p2 = ((n2 + 7) / 8) * 8;
    h->g.cube = (long long)n3 * n1 * h->g.p2;
    const size_t cb = (size_t)h->g.cube * h->esz;
    int rc = GSSTV_OK;
    for (int k = 0; k < 2 && rc == GSSTV_OK; ++k) {
        void** one[] = {&h->u[k], &h->s[k], &h->t[k], &h->y3[k], &h->q[k]};
        for (void** pp : one) if (rc == GSSTV_OK) rc = dalloc(h, pp, cb);
        if (rc == GSSTV_OK) rc = dalloc(h, &h->w1[k], 6 * cb);
        if (rc == GSSTV_OK) rc = dalloc(h, &h->w2[k], 6 * cb);
        if (rc == GSSTV_OK) rc = dalloc(h, &h->y1[k], 2 * cb);
        if (rc == GSSTV_OK) rc = dalloc(h, &h->y2[k], 2 * cb);
    }
    if (rc == GSSTV_OK && cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess) {
        h->cap = nullptr;
        rc = GSSTV_ERR_CUDA;
    }
    if (rc == GSSTV_OK && cudaStreamCreateWithFlags(&h->cap2, cudaStreamNonBlocking) != cudaSuccess) {
        h->cap2 = nullptr;
        rc = GSSTV_ERR_CUDA;
    }
    if (rc == GSSTV_OK) rc = dalloc(h, (void**)&h->v, (size_t)h->g.cube * sizeof(float));
    if (rc == GSSTV_OK) rc = dalloc(h, (void**)&h->sc, sizeof(Scal));
    if (rc == GSSTV_OK && (k1_configure(p->storage) != 0 || light_configure(p->storage) != 0 ||
                           (p->storage == GSSTV_FP32 && k1_tma_configure(p->storage) != 0)))
        rc = GSSTV_ERR_CUDA;
    {
        // The TMA-fed K1 serves float32 storage; 16-bit storage runs the
        // cooperative-load K1.  GSSTV_K1=coop (a debugging aid) selects the
        // cooperative kernel for float32 too.
        const char* ev = std::getenv("GSSTV_K1");
        h->k1_variant = (p->storage == GSSTV_FP32 && !(ev && std::strcmp(ev, "coop") == 0)) ? 1 : 0;
    }
    h->k1_ctas = std::max(k1_grid_ctas(h->g), k1_tma_ctas(h->g));
    h->k2_cap = k2_grid_ctas(h->g);
    if (rc == GSSTV_OK) rc = dalloc(h, (void**)&h->l1.cand[0], kCandCap * sizeof(float));
    if (rc == GSSTV_OK) rc = dalloc(h, (void**)&h->l1.cand[1], kCandCap * sizeof(float));
    if (rc == GSSTV_OK) rc = dalloc(h, (void**)&h->l1.hcnt, 2 * kHistBins * sizeof(unsigned long long));
    if (rc == GSSTV_OK) rc = dalloc(h, (void**)&h->l1.hres, 2 * kHistBins * sizeof(unsigned long long));
    if (rc == GSSTV_OK) rc = dalloc(h, (void**)&h->l1.k1_n, 4 * (size_t)h->k1_ctas * sizeof(unsigned long long));
    if (rc == GSSTV_OK) rc = dalloc(h, (void**)&h->l1.k1_s, 4 * (size_t)h->k1_ctas * sizeof(double));
    if (rc == GSSTV_OK) rc = dalloc(h, (void**)&h->l1.khist, 2 * (size_t)kK1Bins * sizeof(unsigned));
    if (rc == GSSTV_OK) rc = dalloc(h, (void**)&h->l1.nh, 2 * 3 * (size_t)kNarrowBins * sizeof(unsigned));
    if (rc == GSSTV_OK) rc = dalloc(h, (void**)&h->l1.nbinned, 2 * sizeof(unsigned));
    if (rc == GSSTV_OK) rc = dalloc(h, (void**)&h->k2_part, 3 * (size_t)h->k2_cap * sizeof(double));
    if (rc == GSSTV_OK) {
        h->ev.resize(512);
        for (auto& e : h->ev)
            if (rc == GSSTV_OK && cudaEventCreate(&e) != cudaSuccess) { e = nullptr; rc = GSSTV_ERR_CUDA; }
    }
    for (int par = 0; par < 2 && rc == GSSTV_OK && h->k1_variant == 1; ++par) {
        const IterBufs b = bufs(h, par);
        if (k1_tma_maps(p->storage, h->g, b, &h->maps[par]) != 0) rc = GSSTV_ERR_CUDA;
    }
    if (rc == GSSTV_OK) rc = upload_scalars(h, initial_scalars(h->p));
    if (rc != GSSTV_OK) {
        free_all(h);
        delete h;
        return rc;
    }
    *out = h;
    return GSSTV_OK;
}

int gsstv_set_params(gsstv_handle* h, const gsstv_params* p) {
    if (!h) return GSSTV_ERR_ARG;
    TRY(check_params(p));
    if (p->storage != h->p.storage) return GSSTV_ERR_ARG;
    h->p = *p;
    destroy_graphs(h);
    double r[2] = {p->alpha, p->beta};
    TRY(cuda_rc(cudaMemcpyAsync(&h->sc->radius[0], r, sizeof(r), cudaMemcpyHostToDevice, h->st)));
    return cuda_rc(cudaStreamSynchronize(h->st));
}

int gsstv_destroy(gsstv_handle* h) {
    if (!h) return GSSTV_OK;
    free_all(h);
    delete h;
    return GSSTV_OK;
}

int gsstv_load_observation(gsstv_handle* h, const float* d_v) {
    if (!h || !d_v) return GSSTV_ERR_ARG;
    const Geom& g = h->g;
    return cuda_rc(cudaMemcpy2DAsync(h->v, (size_t)g.p2 * 4, d_v, (size_t)g.n2 * 4, (size_t)g.n2 * 4,
                                     (size_t)g.n3 * g.n1, cudaMemcpyDeviceToDevice, h->st));
}

int gsstv_reset_state(gsstv_handle* h) {
    if (!h) return GSSTV_ERR_ARG;
    const size_t cb = (size_t)h->g.cube * h->esz;
    // the standard start in the parity-0 buffers, which the first pass reads;
    // it writes every voxel of the parity-1 buffers before any pass reads
    // them (their padding columns stay zero from the allocation: the passes
    // write zeros there), so those are not cleared
    {
        const int k = 0;
        void* one[] = {h->u[k], h->s[k], h->t[k], h->y3[k], h->q[k]};
        for (void* pp : one) TRY(cuda_rc(cudaMemsetAsync(pp, 0, cb, h->st)));
        TRY(cuda_rc(cudaMemsetAsync(h->w1[k], 0, 6 * cb, h->st)));
        TRY(cuda_rc(cudaMemsetAsync(h->w2[k], 0, 6 * cb, h->st)));
        TRY(cuda_rc(cudaMemsetAsync(h->y1[k], 0, 2 * cb, h->st)));
        TRY(cuda_rc(cudaMemsetAsync(h->y2[k], 0, 2 * cb, h->st)));
    }
    TRY(map_launch(launch_pitched_to_storage(h->p.storage, h->v, h->u[0], h->g, h->st)));
    h->parity = 0;
    return upload_scalars(h, initial_scalars(h->p));
}

int gsstv_iterate(gsstv_handle* h, int n, int* iters_done) {
    if (!h || n < 0) return GSSTV_ERR_ARG;
    if (iters_done) *iters_done = 0;
    int done = 0;
    Scal s;
    if (h->p.tol > 0.0) {
        while (done < n) {
            const int blk = std::min(h->p.check_every, n - done);
            TRY(run_block(h, blk));
            done += blk;
            TRY(flush_timing(h));
            TRY(read_scalars(h, &s));
            TRY(error_of(s));
            h->stats.last_rel_change = s.u2 > 0 ? std::sqrt(s.du2 / s.u2) : INFINITY;
            if (s.u2 > 0 && std::sqrt(s.du2 / s.u2) < h->p.tol) break;
        }
    } else {
        TRY(run_block(h, n));
        done = n;
        TRY(flush_timing(h));
        TRY(read_scalars(h, &s));
        TRY(error_of(s));
        h->stats.last_rel_change = s.u2 > 0 ? std::sqrt(s.du2 / s.u2) : INFINITY;
    }
    h->stats.last_tau_s = s.ctl[0].tau;
    h->stats.last_tau_t = s.ctl[1].tau;
    h->stats.last_l2_scale = s.c[h->parity];
    if (iters_done) *iters_done = done;
    return GSSTV_OK;
}

static bool view_ok(const gsstv_state_view* v) {
    return v && v->u && v->s && v->t && v->w1 && v->w2 && v->y1 && v->y2 && v->y3 && v->y4;
}

// Unpacks the current state into float32 views on the handle's stream (no sync).
static int enqueue_get_state(gsstv_handle* h, const gsstv_state_view* v) {
    const int par = h->parity, sto = h->p.storage;
    {
        const void* src[9] = {h->u[par], h->s[par], h->t[par], h->w1[par], h->w2[par],
                              h->y1[par], h->y2[par], h->y3[par], h->q[par]};
        float* dst[9] = {v->u, v->s, v->t, v->w1, v->w2, v->y1, v->y2, v->y3, v->y4};
        const int rc = launch_unpack_state(sto, src, dst, &h->sc->c[par], h->g, h->st);
        if (rc == 0) return GSSTV_OK;
        if (rc != 1) return GSSTV_ERR_CUDA;
    }
    TRY(map_launch(launch_unpack(sto, h->u[par], v->u, h->g, 1, h->st)));
    TRY(map_launch(launch_unpack(sto, h->s[par], v->s, h->g, 1, h->st)));
    TRY(map_launch(launch_unpack(sto, h->t[par], v->t, h->g, 1, h->st)));
    TRY(map_launch(launch_unpack(sto, h->w1[par], v->w1, h->g, 6, h->st)));
    TRY(map_launch(launch_unpack(sto, h->w2[par], v->w2, h->g, 6, h->st)));
    TRY(map_launch(launch_unpack(sto, h->y1[par], v->y1, h->g, 2, h->st)));
    TRY(map_launch(launch_unpack(sto, h->y2[par], v->y2, h->g, 2, h->st)));
    TRY(map_launch(launch_unpack(sto, h->y3[par], v->y3, h->g, 1, h->st)));
    return map_launch(launch_scale_unpack(sto, h->q[par], &h->sc->c[par], v->y4, h->g, h->st));
}

static int copy_out_device(gsstv_handle* h, float* d_u, float* d_s, float* d_t) {
    const int par = h->parity;
    if (d_u) TRY(map_launch(launch_unpack(h->p.storage, h->u[par], d_u, h->g, 1, h->st)));
    if (d_s) TRY(map_launch(launch_unpack(h->p.storage, h->s[par], d_s, h->g, 1, h->st)));
    if (d_t) TRY(map_launch(launch_unpack(h->p.storage, h->t[par], d_t, h->g, 1, h->st)));
    return cuda_rc(cudaStreamSynchronize(h->st));
}

int gsstv_solve(gsstv_handle* h, const float* d_v, float* d_u, float* d_s, float* d_t, int* iters_done) {
    if (!h || !d_v || !d_u) return GSSTV_ERR_ARG;
    TRY(gsstv_load_observation(h, d_v));
    TRY(gsstv_reset_state(h));
    TRY(gsstv_iterate(h, h->p.max_iter, iters_done));
    return copy_out_device(h, d_u, d_s, d_t);
}

int gsstv_solve_host(gsstv_handle* h, const float* h_v, float* h_u, float* h_s, float* h_t, int* iters_done) {
    if (!h || !h_v || !h_u) return GSSTV_ERR_ARG;
    const Geom& g = h->g;
    const size_t w = (size_t)g.n2 * 4, dp = (size_t)g.p2 * 4, rows = (size_t)g.n3 * g.n1;
    // rows without padding (N2 a multiple of 8) copy as one block
    if (dp == w)
        TRY(cuda_rc(cudaMemcpyAsync(h->v, h_v, w * rows, cudaMemcpyHostToDevice, h->st)));
    else
        TRY(cuda_rc(cudaMemcpy2DAsync(h->v, dp, h_v, w, w, rows, cudaMemcpyHostToDevice, h->st)));
    TRY(gsstv_reset_state(h));
    TRY(gsstv_iterate(h, h->p.max_iter, iters_done));
    const int par = h->parity;
    void* src[3] = {h->u[par], h->s[par], h->t[par]};
    float* dst[3] = {h_u, h_s, h_t};
    if (h->p.storage != GSSTV_FP32 && !h->tmp) {
        void* t = nullptr;
        TRY(dalloc(h, &t, (size_t)g.n3 * g.n1 * g.n2 * 4));
        h->tmp = (float*)t;
    }
    for (int k = 0; k < 3; ++k) {
        if (!dst[k]) continue;
        if (h->p.storage == GSSTV_FP32 && dp == w) {
            TRY(cuda_rc(cudaMemcpyAsync(dst[k], src[k], w * rows, cudaMemcpyDeviceToHost, h->st)));
        } else if (h->p.storage == GSSTV_FP32) {
            TRY(cuda_rc(cudaMemcpy2DAsync(dst[k], w, src[k], dp, w, rows, cudaMemcpyDeviceToHost, h->st)));
        } else {
            TRY(map_launch(launch_unpack(h->p.storage, src[k], h->tmp, g, 1, h->st)));
            TRY(cuda_rc(cudaMemcpyAsync(dst[k], h->tmp, w * rows, cudaMemcpyDeviceToHost, h->st)));
        }
    }
    return cuda_rc(cudaStreamSynchronize(h->st));
}

int gsstv_get_state(gsstv_handle* h, const gsstv_state_view* v) {
    if (!h || !view_ok(v)) return GSSTV_ERR_ARG;
    TRY(enqueue_get_state(h, v));
    return cuda_rc(cudaStreamSynchronize(h->st));
}

int gsstv_set_state(gsstv_handle* h, const gsstv_state_view* v) {
    if (!h || !view_ok(v)) return GSSTV_ERR_ARG;
    const int par = h->parity, sto = h->p.storage;
    TRY(map_launch(launch_pack(sto, v->u, h->u[par], h->g, 1, h->st)));
    TRY(map_launch(launch_pack(sto, v->s, h->s[par], h->g, 1, h->st)));
    TRY(map_launch(launch_pack(sto, v->t, h->t[par], h->g, 1, h->st)));
    TRY(map_launch(launch_pack(sto, v->w1, h->w1[par], h->g, 6, h->st)));
    TRY(map_launch(launch_pack(sto, v->w2, h->w2[par], h->g, 6, h->st)));
    TRY(map_launch(launch_pack(sto, v->y1, h->y1[par], h->g, 2, h->st)));
    TRY(map_launch(launch_pack(sto, v->y2, h->y2[par], h->g, 2, h->st)));
    TRY(map_launch(launch_pack(sto, v->y3, h->y3[par], h->g, 1, h->st)));
    TRY(map_launch(launch_pack(sto, v->y4, h->q[par], h->g, 1, h->st)));
    // y4 is now stored unscaled (c = 0); the threshold search starts afresh
    return upload_scalars(h, initial_scalars(h->p));
}

int gsstv_autotune(gsstv_handle* h, int passes, int* chunk_out) {
    if (chunk_out) *chunk_out = 0;
    if (!h || passes < 1) return GSSTV_ERR_ARG;
    if (h->k1_variant != 1) return GSSTV_OK;          // the cooperative kernel has no run length to tune
    int cand[6];
    const int nc = k1_tma_chunk_candidates(h->g, cand, 6);
    const gsstv_stats saved_stats = h->stats;
    const int saved_timing = h->timing;
    double best = INFINITY;
    int best_chunk = 0;
    int rc = flush_timing(h);
    for (int k = 0; k < nc && rc == GSSTV_OK; ++k) {
        h->k1_chunk = cand[k];
        h->timing = 0;
        rc = gsstv_reset_state(h);
        if (rc == GSSTV_OK) rc = run_block(h, 1);     // untimed first pass
        h->timing = 1;
        const double ms0 = h->stats.k1_ms;
        const int64_t n0 = h->stats.k1_launches;
        if (rc == GSSTV_OK) rc = run_block(h, passes);
        if (rc == GSSTV_OK) rc = flush_timing(h);
        Scal sc;
        if (rc == GSSTV_OK) rc = read_scalars(h, &sc);
        if (rc == GSSTV_OK) rc = error_of(sc);
        const int64_t n = h->stats.k1_launches - n0;
        if (rc == GSSTV_OK && n > 0) {
            const double ms = (h->stats.k1_ms - ms0) / (double)n;
            if (ms < best) { best = ms; best_chunk = cand[k]; }
        }
    }
    h->timing = saved_timing;
    h->stats = saved_stats;
    h->k1_chunk = rc == GSSTV_OK ? best_chunk : 0;
    destroy_graphs(h);                                  // graphs hold the old launch shape
    TRY(rc);
    TRY(gsstv_reset_state(h));
    if (chunk_out) *chunk_out = h->k1_chunk;
    return GSSTV_OK;
}

int gsstv_get_stats(gsstv_handle* h, gsstv_stats* out) {
    if (!h || !out) return GSSTV_ERR_ARG;
    TRY(flush_timing(h));
    Scal s;
    TRY(read_scalars(h, &s));
    *out = h->stats;
    out->tau_window_hits = s.ctl[0].hits + s.ctl[1].hits;
    out->tau_exact_runs = s.ctl[0].exact_runs + s.ctl[1].exact_runs;
    out->tau_retry_hits = s.ctl[0].retry_hits + s.ctl[1].retry_hits;
    out->search_passes = s.gate_opens;
    return GSSTV_OK;
}

int gsstv_reset_stats(gsstv_handle* h) {
    if (!h) return GSSTV_ERR_ARG;
    TRY(flush_timing(h));
    h->stats = gsstv_stats{};
    Scal s;
    TRY(read_scalars(h, &s));
    for (int v = 0; v < 2; ++v) { s.ctl[v].hits = 0; s.ctl[v].exact_runs = 0; s.ctl[v].retry_hits = 0; }
    s.gate_opens = 0;
    return upload_scalars(h, s);
}

int gsstv_set_timing(gsstv_handle* h, int on) {
    if (!h) return GSSTV_ERR_ARG;
    TRY(flush_timing(h));
    h->timing = on ? 1 : 0;
    // build the timed graphs of the current parity now, so that timed passes
    // do not wait for them
    const int G = h->p.graph_iters > 0 ? ((h->p.graph_iters + 1) / 2) * 2 : 0;
    if (on && G > 0 && 2 * G * gsstv_handle::kTimedSlots <= (int)h->ev.size()) {
        if (h->timed_len != G) destroy_graphs(h);
        h->timed_len = G;
        for (int k = 0; k < gsstv_handle::kTimedSlots; ++k) {
            h->ev_used = 2 * G * k;
            if (!h->timed_exec[h->parity][k]) TRY(build_graph_exec(h, h->parity, G, true, &h->timed_exec[h->parity][k]));
        }
        h->ev_used = 0;
    }
    return GSSTV_OK;
}

int64_t gsstv_device_bytes(const gsstv_handle* h) { return h ? h->bytes : 0; }

int gsstv_project_l1ball(const float* d_x, int64_t n, double radius, float* d_out, double* tau_out,
                         void* stream) {
    if (!d_x || !d_out || n < 0 || !(radius >= 0.0) || !std::isfinite(radius)) return GSSTV_ERR_ARG;
    if (n == 0) { if (tau_out) *tau_out = 0.0; return GSSTV_OK; }
    const int rc = l1_project_standalone(d_x, (long long)n, radius, d_out, tau_out, (cudaStream_t)stream);
    return rc == 0 ? GSSTV_OK : rc == -2 ? GSSTV_ERR_OOM : rc == -6 ? GSSTV_ERR_INTERNAL : GSSTV_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// reverse mode: vector-Jacobian products of the iteration
// ---------------------------------------------------------------------------
// One pass transposed (gsstv_vjp_step) and the adjoint of a whole run of K
// passes from the standard start (gsstv_unrolled_vjp): the forward run keeps
// a checkpoint every C passes, the reverse sweep re-runs each segment from
// its checkpoint, keeps that segment's states and applies the one-pass
// transpose to them from the last to the first.
namespace {

constexpr int kStateCubes = 21;   // u, s, t, w1 (6), w2 (6), y1 (2), y2 (2), y3, y4

// views into one state of kStateCubes * P floats (P = adj_stride(N): every
// field on a 256-byte boundary; the planes of w1, w2, y1, y2 at stride N)
gsstv_state_view state_at(float* base, long long P) {
    gsstv_state_view v;
    v.u = base; v.s = base + P; v.t = base + 2 * P; v.w1 = base + 3 * P; v.w2 = base + 9 * P;
    v.y1 = base + 15 * P; v.y2 = base + 17 * P; v.y3 = base + 19 * P; v.y4 = base + 20 * P;
    return v;
}

void view_ptrs(const gsstv_state_view* v, float* out[9]) {
    out[0] = v->u; out[1] = v->s; out[2] = v->t; out[3] = v->w1; out[4] = v->w2;
    out[5] = v->y1; out[6] = v->y2; out[7] = v->y3; out[8] = v->y4;
}

int vjp_launch(gsstv_handle* h, const gsstv_state_view* x, const gsstv_state_view* x1,
               const gsstv_state_view* b1, const gsstv_state_view* bo, float* vbar, double* d_pbar,
               void* work) {
    const gsstv_params& p = h->p;
    const double prm[16] = {p.gamma_u, p.gamma_w1, p.gamma_w2, p.gamma_s, p.gamma_t,
                            p.gamma_y1, p.gamma_y2, p.gamma_y3, p.gamma_y4,
                            p.gamma_w1 * p.omega, p.gamma_w2, p.mu_lo, p.mu_hi, p.eps, p.alpha, p.beta};
    float *xa[9], *x1a[9], *b1a[9], *boa[9];
    view_ptrs(x, xa); view_ptrs(x1, x1a); view_ptrs(b1, b1a); view_ptrs(bo, boa);
    const Geom& g = h->g;
    return map_launch(launch_adjoint_step(g.n1, g.n2, g.n3, xa, x1a, b1a, boa, h->v, g.p2, vbar, d_pbar,
                                          work, prm, h->st));
}

// device scratch of one gsstv_unrolled_vjp call, released on every return
struct Scratch {
    void* p = nullptr;
    ~Scratch() { if (p) cudaFree(p); }
};

}  // namespace

int gsstv_vjp_step(gsstv_handle* h, const gsstv_state_view* x, const gsstv_state_view* x_next,
                   const gsstv_state_view* bar_next, const gsstv_state_view* bar, float* d_vbar,
                   double* h_pbar) {
    if (!h || !view_ok(x) || !view_ok(x_next) || !view_ok(bar_next) || !view_ok(bar) || !d_vbar)
        return GSSTV_ERR_ARG;
    if (h->p.storage != GSSTV_FP32) return GSSTV_ERR_ARG;
    const long long n = (long long)h->g.n1 * h->g.n2 * h->g.n3;
    const size_t wb = adjoint_workspace_bytes(n);
    if (!h->adj_work) TRY(dalloc(h, &h->adj_work, wb + 4 * sizeof(double)));
    double* d_pbar = (double*)((char*)h->adj_work + wb);
    TRY(cuda_rc(cudaMemsetAsync(d_pbar, 0, 4 * sizeof(double), h->st)));
    TRY(vjp_launch(h, x, x_next, bar_next, bar, d_vbar, d_pbar, h->adj_work));
    if (!h_pbar) return GSSTV_OK;
    double pb[4];
    TRY(cuda_rc(cudaMemcpyAsync(pb, d_pbar, sizeof(pb), cudaMemcpyDeviceToHost, h->st)));
    TRY(cuda_rc(cudaStreamSynchronize(h->st)));
    for (int k = 0; k < 4; ++k) h_pbar[k] += pb[k];
    return GSSTV_OK;
}

int gsstv_unrolled_vjp(gsstv_handle* h, int iters, int ckpt_every, const float* d_ubar, float* d_vbar,
                       double* h_pbar) {
    if (!h || iters < 0 || ckpt_every < 0 || !d_ubar || !d_vbar || !h_pbar) return GSSTV_ERR_ARG;
    if (h->p.storage != GSSTV_FP32) return GSSTV_ERR_ARG;
    const long long n = (long long)h->g.n1 * h->g.n2 * h->g.n3;
    const size_t cube = (size_t)n * sizeof(float);
    for (int k = 0; k < 4; ++k) h_pbar[k] = 0.0;
    if (iters == 0) {   // u_0 = v
        TRY(cuda_rc(cudaMemcpyAsync(d_vbar, d_ubar, cube, cudaMemcpyDeviceToDevice, h->st)));
        return cuda_rc(cudaStreamSynchronize(h->st));
    }
    const int C = ckpt_every > 0 ? std::min(ckpt_every, iters)
                                 : std::max(1, (int)std::ceil(std::sqrt((double)iters)));
    const int nck = (iters + C - 1) / C;
    const long long P = adj_stride(n);
    const size_t sbytes = (size_t)kStateCubes * P * sizeof(float);
    const size_t wb = adjoint_workspace_bytes(n);
    // nck checkpoints, C segment states, the adjoint state, the workspace
    Scratch scr;
    if (cudaMalloc(&scr.p, (size_t)(nck + C + 1) * sbytes + wb + 4 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        scr.p = nullptr;
        return GSSTV_ERR_OOM;
    }
    float* base = (float*)scr.p;
    auto slot = [&](int k) { return state_at(base + (size_t)k * kStateCubes * P, P); };
    const gsstv_state_view bar = slot(nck + C);
    void* work = base + (size_t)(nck + C + 1) * kStateCubes * P;
    double* d_pbar = (double*)((char*)work + wb);
    // forward: the state at the start of every segment.  With a checkpoint
    // every pass (C = 1) the forward keeps every state, the last one in the
    // (otherwise unused) first segment slot, and the sweep re-runs nothing;
    // otherwise the last segment needs no run here.
    const bool keep_all = C == 1;
    TRY(gsstv_reset_state(h));
    for (int c = 0; c < nck; ++c) {
        const gsstv_state_view v = slot(c);
        TRY(enqueue_get_state(h, &v));
        if (c + 1 < nck || keep_all) TRY(run_block(h, C));
    }
    if (keep_all) {
        const gsstv_state_view v = slot(nck);
        TRY(enqueue_get_state(h, &v));
    }
    TRY(flush_timing(h));
    Scal sc;
    TRY(read_scalars(h, &sc));
    TRY(error_of(sc));
    // reverse sweep, the adjoint transposed in place
    TRY(cuda_rc(cudaMemsetAsync(bar.u, 0, sbytes, h->st)));
    TRY(cuda_rc(cudaMemcpyAsync(bar.u, d_ubar, cube, cudaMemcpyDeviceToDevice, h->st)));
    TRY(cuda_rc(cudaMemsetAsync(d_vbar, 0, cube, h->st)));
    TRY(cuda_rc(cudaMemsetAsync(d_pbar, 0, 4 * sizeof(double), h->st)));
    if (keep_all) {
        for (int k = iters - 1; k >= 0; --k) {
            const gsstv_state_view xk = slot(k), xk1 = slot(k + 1);
            TRY(vjp_launch(h, &xk, &xk1, &bar, &bar, d_vbar, d_pbar, work));
        }
    }
    for (int c = keep_all ? -1 : nck - 1; c >= 0; --c) {
        const int len = std::min(C, iters - c * C);
        const gsstv_state_view start = slot(c);
        TRY(gsstv_set_state(h, &start));
        for (int j = 1; j <= len; ++j) {             // segment state j in slot nck + j - 1
            TRY(run_block(h, 1));
            const gsstv_state_view v = slot(nck + j - 1);
            TRY(enqueue_get_state(h, &v));
        }
        TRY(flush_timing(h));
        TRY(read_scalars(h, &sc));
        TRY(error_of(sc));
        for (int j = len - 1; j >= 0; --j) {
            const gsstv_state_view xj = j == 0 ? start : slot(nck + j - 1);
            const gsstv_state_view xj1 = slot(nck + j);
            TRY(vjp_launch(h, &xj, &xj1, &bar, &bar, d_vbar, d_pbar, work));
        }
    }
    // the start u = v
    TRY(map_launch(launch_axpy(d_vbar, bar.u, 1.0f, n, h->st)));
    double pb[4];
    TRY(cuda_rc(cudaMemcpyAsync(pb, d_pbar, sizeof(pb), cudaMemcpyDeviceToHost, h->st)));
    TRY(cuda_rc(cudaStreamSynchronize(h->st)));
    for (int k = 0; k < 4; ++k) h_pbar[k] = pb[k];
    return GSSTV_OK;
}

// ---------------------------------------------------------------------------
// batches of independent cubes
// ---------------------------------------------------------------------------
// Each cube keeps a handle of its own on a stream of its own; a solve keeps
// one block of iterations in flight per unfinished cube (CUDA graphs, as for a
// single handle), reads each block's scalars back asynchronously and decides
// the cube's stopping rule (Eq. 28) on the host as gsstv_iterate does, so a
// cube's result is the one gsstv_solve gives it alone.  Small cubes are
// launch-bound; running many at once fills the GPU.
struct gsstv_batch {
    std::vector<gsstv_handle*> h;
    std::vector<cudaStream_t> st;
    std::vector<cudaEvent_t> ev;
    Scal* pinned = nullptr;        // one Scal per cube, page-locked
    cudaStream_t caller = nullptr;
    // one launch per stage for every cube (float32 cubes, at most kBatchMax)
    bool fused = false;
    K1Maps* dmaps = nullptr;       // [cube][parity] tensor maps in device memory
    int* live = nullptr;           // device: cubes still iterating
    int* live_host = nullptr;      // page-locked copy
    cudaStream_t cap = nullptr;    // private capture stream
    cudaStream_t cap2 = nullptr;   // and one for the bodies of conditional graph nodes
    cudaGraphExec_t gexec = nullptr;
    int graph_len = 0;
    std::vector<int> graph_chunks;  // the cubes' K1 band runs the graph was built with
    std::vector<int> graph_set;     // and the cubes it runs
};

int gsstv_batch_destroy(gsstv_batch* b) {
    if (!b) return GSSTV_OK;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->caller) cudaStreamSynchronize(b->caller);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->cap2) cudaStreamDestroy(b->cap2);
    if (b->dmaps) cudaFree(b->dmaps);
    if (b->live) cudaFree(b->live);
    if (b->live_host) cudaFreeHost(b->live_host);
    for (gsstv_handle* h : b->h) gsstv_destroy(h);
    for (cudaEvent_t e : b->ev) if (e) cudaEventDestroy(e);
    for (cudaStream_t s : b->st) if (s) cudaStreamDestroy(s);
    if (b->pinned) cudaFreeHost(b->pinned);
    delete b;
    return GSSTV_OK;
}

int gsstv_batch_create(gsstv_batch** out, int ncubes, const int* n1, const int* n2, const int* n3,
                       const gsstv_params* params, void* stream) {
    if (!out) return GSSTV_ERR_ARG;
    *out = nullptr;
    if (ncubes < 1 || !n1 || !n2 || !n3 || !params) return GSSTV_ERR_ARG;
    for (int c = 0; c < ncubes; ++c) {
        if (!shape_ok(n1[c], n2[c], n3[c])) return GSSTV_ERR_ARG;
        TRY(check_params(&params[c]));
    }
    gsstv_batch* b = new gsstv_batch();
    b->caller = (cudaStream_t)stream;
    int rc = GSSTV_OK;
    if (cudaMallocHost((void**)&b->pinned, sizeof(Scal) * ncubes) != cudaSuccess) {
        b->pinned = nullptr;
        rc = GSSTV_ERR_OOM;
    }
    for (int c = 0; c < ncubes && rc == GSSTV_OK; ++c) {
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) { rc = GSSTV_ERR_CUDA; break; }
        b->st.push_back(s);
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) { rc = GSSTV_ERR_CUDA; break; }
        b->ev.push_back(e);
        gsstv_handle* h = nullptr;
        rc = gsstv_create(&h, n1[c], n2[c], n3[c], &params[c], s);
        if (rc == GSSTV_OK) b->h.push_back(h);
    }
    // Float32 cubes run every stage of a pass as one launch over all cubes
    // (GSSTV_BATCH=streams keeps one stream per cube, as 16-bit cubes do).
    if (rc == GSSTV_OK) {
        const char* ev = std::getenv("GSSTV_BATCH");
        b->fused = ncubes <= kBatchMax && !(ev && std::strcmp(ev, "streams") == 0);
        for (gsstv_handle* h : b->h)
            if (h->p.storage != GSSTV_FP32 || h->k1_variant != 1) b->fused = false;
    }
    if (rc == GSSTV_OK && b->fused) {
        if (batch_configure() != 0) rc = GSSTV_ERR_CUDA;
        if (rc == GSSTV_OK && cudaMalloc((void**)&b->dmaps, sizeof(K1Maps) * 2 * ncubes) != cudaSuccess) {
            cudaGetLastError();
            b->dmaps = nullptr;
            rc = GSSTV_ERR_OOM;
        }
        if (rc == GSSTV_OK && cudaMalloc((void**)&b->live, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            b->live = nullptr;
            rc = GSSTV_ERR_OOM;
        }
        if (rc == GSSTV_OK && cudaMallocHost((void**)&b->live_host, sizeof(int)) != cudaSuccess) {
            b->live_host = nullptr;
            rc = GSSTV_ERR_OOM;
        }
        if (rc == GSSTV_OK && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
            b->cap = nullptr;
            rc = GSSTV_ERR_CUDA;
        }
        if (rc == GSSTV_OK && cudaStreamCreateWithFlags(&b->cap2, cudaStreamNonBlocking) != cudaSuccess) {
            b->cap2 = nullptr;
            rc = GSSTV_ERR_CUDA;
        }
        for (int c = 0; c < ncubes && rc == GSSTV_OK; ++c)
            rc = cuda_rc(cudaMemcpy(b->dmaps + 2 * c, b->h[c]->maps, 2 * sizeof(K1Maps), cudaMemcpyHostToDevice));
    }
    if (rc != GSSTV_OK) { gsstv_batch_destroy(b); return rc; }
    *out = b;
    return GSSTV_OK;
}

int gsstv_batch_size(const gsstv_batch* b) { return b ? (int)b->h.size() : 0; }

namespace {

// One pass of the cubes in `set` from parity `par`: each stage one launch
// (a cube that has stopped returns at once from each).
int batch_enqueue(gsstv_batch* b, const std::vector<int>& set, int par, cudaStream_t st) {
    const int nc = (int)set.size();
    BatchCube cubes[kBatchMax];
    for (int k = 0; k < nc; ++k) {
        const int c = set[k];
        gsstv_handle* h = b->h[c];
        BatchCube& q = cubes[k];
        q.g = h->g;
        q.b = bufs(h, par);
        q.p = iparams(h, par);
        q.p.max_iter = h->p.max_iter;          // the stopping rule on the device
        q.p.tol = h->p.tol;
        q.p.check_every = h->p.check_every;
        q.p.live = b->live;
        q.sc = h->sc;
        q.l1 = h->l1;
        q.k2_part = h->k2_part;
        q.k2_cap = h->k2_cap;
        q.k1_chunk = h->k1_chunk;
        q.k1_ctas = h->k1_ctas;
        q.maps = b->dmaps + 2 * c + par;
    }
    TRY(map_launch(launch_k1_batch(cubes, nc, st)));
    // K1's window finish, then the search launches behind a conditional node
    // that it opens (the fused solve is always captured)
    auto k1_finish = [&](cudaGraphConditionalHandle c) -> int {
        return map_launch(launch_finish_batch(cubes, nc, 2, st, 1, c));
    };
    TRY(capture_if_search(st, b->cap2, k1_finish, [&](cudaStream_t q) -> int {
        TRY(map_launch(launch_window_batch(cubes, nc, q)));
        TRY(map_launch(launch_finish_batch(cubes, nc, 0, q)));
        for (int level = 0; level < 3; ++level) TRY(map_launch(launch_radix_batch(cubes, nc, level, q)));
        TRY(map_launch(launch_gather_batch(cubes, nc, q)));
        TRY(map_launch(launch_finish_batch(cubes, nc, 1, q)));
        return GSSTV_OK;
    }));
    TRY(map_launch(launch_k2_batch(cubes, nc, st)));
    return GSSTV_OK;
}

// The graph of G passes over the cubes in `set` (rebuilt only when the set
// or a cube's K1 band run has changed).
int batch_graph(gsstv_batch* b, const std::vector<int>& set, int G) {
    std::vector<int> chunks;
    for (int c : set) chunks.push_back(b->h[c]->k1_chunk);   // (the autotuner may change them)
    if (b->gexec && b->graph_len == G && chunks == b->graph_chunks && set == b->graph_set) return GSSTV_OK;
    if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
    cudaGraph_t graph = nullptr;
    TRY(cuda_rc(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal)));
    int rc = GSSTV_OK;
    for (int k = 0; k < G && rc == GSSTV_OK; ++k) rc = batch_enqueue(b, set, k & 1, b->cap);
    const cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
    if (rc != GSSTV_OK) { if (graph) cudaGraphDestroy(graph); return rc; }
    TRY(cuda_rc(e));
    const cudaError_t ei = cudaGraphInstantiate(&b->gexec, graph, 0);
    cudaGraphDestroy(graph);
    TRY(cuda_rc(ei));
    b->graph_len = G;
    b->graph_chunks = chunks;
    b->graph_set = set;
    return GSSTV_OK;
}

// The fused solve: every cube from its standard start, blocks of passes as
// one CUDA graph (even length: the parity comes back to 0) until no cube is
// left iterating.  A cube stops on the device at the pass its own stopping
// rule names, exactly as gsstv_iterate stops it (Eq. 28 every check_every
// passes, or max_iter).  After a block in which cubes stopped, the graph is
// rebuilt over the cubes still iterating, so that stopped cubes stop costing
// launches; they all sit at parity 0 then, having run every pass so far.
int batch_solve_fused(gsstv_batch* b, const float* const* d_v, float* const* d_u, float* const* d_s,
                      float* const* d_t, int* iters_done) {
    const int nc = (int)b->h.size();
    int live = 0, most = 0;
    std::vector<int> set;
    for (int c = 0; c < nc; ++c) {
        gsstv_handle* h = b->h[c];
        TRY(gsstv_load_observation(h, d_v[c]));
        TRY(gsstv_reset_state(h));                       // synchronises the cube's stream
        if (h->p.max_iter > 0) {
            ++live;
            most = std::max(most, h->p.max_iter);
            set.push_back(c);
        } else {                                         // nothing to run: stopped at the start
            const int one[2] = {1, 0};
            TRY(cuda_rc(cudaMemcpy(&h->sc->done, one, sizeof(one), cudaMemcpyHostToDevice)));
        }
    }
    TRY(cuda_rc(cudaMemcpyAsync(b->live, &live, sizeof(int), cudaMemcpyHostToDevice, b->caller)));
    const int G = 16;
    for (int run = 0; live > 0 && run < most; run += G) {
        if (live < (int)set.size()) {
            // which cubes stopped in the last block (their done flags)
            for (int c : set)
                TRY(cuda_rc(cudaMemcpyAsync(&b->pinned[c].done, &b->h[c]->sc->done, sizeof(int),
                                            cudaMemcpyDeviceToHost, b->caller)));
            TRY(cuda_rc(cudaStreamSynchronize(b->caller)));
            std::vector<int> keep;
            for (int c : set)
                if (!b->pinned[c].done) keep.push_back(c);
            set.swap(keep);
            if (set.empty()) break;
        }
        TRY(batch_graph(b, set, G));
        TRY(cuda_rc(cudaGraphLaunch(b->gexec, b->caller)));
        TRY(cuda_rc(cudaMemcpyAsync(b->live_host, b->live, sizeof(int), cudaMemcpyDeviceToHost, b->caller)));
        TRY(cuda_rc(cudaStreamSynchronize(b->caller)));
        live = *b->live_host;
    }
    int rc = GSSTV_OK;
    for (int c = 0; c < nc && rc == GSSTV_OK; ++c) {
        gsstv_handle* h = b->h[c];
        Scal s;
        rc = read_scalars(h, &s);
        if (rc == GSSTV_OK) rc = error_of(s);
        if (rc != GSSTV_OK) break;
        h->parity = s.done ? s.stop_parity : 0;
        h->stats.iterations += s.iter;
        h->stats.last_rel_change = s.u2 > 0 ? std::sqrt(s.du2 / s.u2) : INFINITY;
        h->stats.last_tau_s = s.ctl[0].tau;
        h->stats.last_tau_t = s.ctl[1].tau;
        h->stats.last_l2_scale = s.c[h->parity];
        if (iters_done) iters_done[c] = (int)s.iter;
        rc = copy_out_device(h, d_u[c], d_s ? d_s[c] : nullptr, d_t ? d_t[c] : nullptr);
    }
    return rc;
}

}  // namespace

int gsstv_batch_solve(gsstv_batch* b, const float* const* d_v, float* const* d_u, float* const* d_s,
                      float* const* d_t, int* iters_done) {
    if (!b || !d_v || !d_u) return GSSTV_ERR_ARG;
    const int nc = (int)b->h.size();
    for (int c = 0; c < nc; ++c) if (!d_v[c] || !d_u[c]) return GSSTV_ERR_ARG;
    // the inputs were written on the caller's stream
    TRY(cuda_rc(cudaStreamSynchronize(b->caller)));
    if (b->fused) return batch_solve_fused(b, d_v, d_u, d_s, d_t, iters_done);
    std::vector<int> done(nc, 0), left(nc, 0), busy(nc, 0), over(nc, 0);
    int rc = GSSTV_OK;
    auto launch_block = [&](int c) {
        gsstv_handle* h = b->h[c];
        const int blk = h->p.tol > 0.0 ? std::min(h->p.check_every, left[c]) : left[c];
        TRY(run_block(h, blk));
        left[c] -= blk;
        done[c] += blk;
        TRY(cuda_rc(cudaMemcpyAsync(&b->pinned[c], h->sc, sizeof(Scal), cudaMemcpyDeviceToHost, h->st)));
        TRY(cuda_rc(cudaEventRecord(b->ev[c], h->st)));
        busy[c] = 1;
        return GSSTV_OK;
    };
    for (int c = 0; c < nc && rc == GSSTV_OK; ++c) {
        gsstv_handle* h = b->h[c];
        rc = gsstv_load_observation(h, d_v[c]);
        if (rc == GSSTV_OK) rc = gsstv_reset_state(h);
        left[c] = h->p.max_iter;
        if (rc == GSSTV_OK) {
            if (left[c] > 0) rc = launch_block(c);
            else over[c] = 1;
        }
    }
    int remaining = 0;
    for (int c = 0; c < nc; ++c) remaining += over[c] ? 0 : 1;
    while (rc == GSSTV_OK && remaining > 0) {
        bool progress = false;
        for (int c = 0; c < nc && rc == GSSTV_OK; ++c) {
            if (over[c] || !busy[c]) continue;
            const cudaError_t q = cudaEventQuery(b->ev[c]);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) { rc = GSSTV_ERR_CUDA; break; }
            progress = true;
            busy[c] = 0;
            gsstv_handle* h = b->h[c];
            const Scal& s = b->pinned[c];
            rc = error_of(s);
            if (rc != GSSTV_OK) break;
            const double rel = s.u2 > 0 ? std::sqrt(s.du2 / s.u2) : INFINITY;
            h->stats.last_rel_change = rel;
            const bool converged = h->p.tol > 0.0 && s.u2 > 0 && rel < h->p.tol;
            if (converged || left[c] == 0) {
                h->stats.last_tau_s = s.ctl[0].tau;
                h->stats.last_tau_t = s.ctl[1].tau;
                h->stats.last_l2_scale = s.c[h->parity];
                over[c] = 1;
                --remaining;
            } else {
                rc = launch_block(c);
            }
        }
        if (!progress && rc == GSSTV_OK) std::this_thread::yield();
    }
    for (int c = 0; c < nc && rc == GSSTV_OK; ++c) {
        if (iters_done) iters_done[c] = done[c];
        rc = copy_out_device(b->h[c], d_u[c], d_s ? d_s[c] : nullptr, d_t ? d_t[c] : nullptr);
    }
    // leave no work of the batch in flight on an error
    for (cudaStream_t s : b->st) cudaStreamSynchronize(s);
    return rc;
}

int gsstv_batch_handle(gsstv_batch* b, int c, gsstv_handle** out) {
    if (!b || !out || c < 0 || c >= (int)b->h.size()) return GSSTV_ERR_ARG;
    *out = b->h[c];
    return GSSTV_OK;
}

// ---------------------------------------------------------------------------
// one cube stored as band slabs
// ---------------------------------------------------------------------------
// The cube's bands are split into S contiguous slabs, each kept in allocations
// of its own with one halo band on each side (only D_s and D_s^T couple
// bands, Sec. II-A).  A pass runs every stage of the single-handle pass on
// each slab in turn; the global sums of a stage (l1 window statistics,
// histograms and candidates, radix histograms, the l2-ball and Eq. 28 norms)
// go to one shared reduction area and are finished once for all slabs (by the
// finishing launch after the stage, or by the last CTA of all the stage's
// launches).  After the pass the halos are refreshed with one copy per
// plane: the band above a slab (u, q, y1, y2: what the next pass's u' of that
// band needs) and the band below it (y2: D^T y2 there, for D_s^T).  This is
// the data flow of a cube split over several GPUs, with the shared reduction
// area standing in for all-reduces of the partial sums and the copies for the
// halo exchange.
struct gsstv_slabs {
    int n1 = 0, n2 = 0, n3 = 0, S = 0;
    gsstv_params p{};
    cudaStream_t st = nullptr;
    cudaStream_t cap = nullptr;
    cudaStream_t cap2 = nullptr;
    std::vector<gsstv_handle*> h;        // slab storage: bands [L0, L0 + h->g.n3) of the cube
    std::vector<int> B0, B1, L0;         // owned bands [B0, B1), first stored band L0
    std::vector<SlabPart> k1p, winp, radp, gatp, k2p;
    std::vector<int> k1_chunk;
    Scal* sc = nullptr;
    L1Work l1{};
    double* k2_part = nullptr;
    int k2_cap = 0, win_cap = 0;
    std::vector<void*> allocs;
    int parity = 0;
    cudaGraphExec_t gexec[2]{};
    int graph_len = 0;
    gsstv_stats stats{};
};

namespace {

int slabs_alloc(gsstv_slabs* G, void** out, size_t bytes) {
    *out = nullptr;
    if (cudaMalloc(out, std::max<size_t>(bytes, 16)) != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        return GSSTV_ERR_OOM;
    }
    G->allocs.push_back(*out);
    return cuda_rc(cudaMemsetAsync(*out, 0, std::max<size_t>(bytes, 16), G->st));
}

void slabs_free(gsstv_slabs* G) {
    for (int k = 0; k < 2; ++k)
        if (G->gexec[k]) { cudaGraphExecDestroy(G->gexec[k]); G->gexec[k] = nullptr; }
    if (G->st) cudaStreamSynchronize(G->st);
    if (G->cap) { cudaStreamDestroy(G->cap); G->cap = nullptr; }
    if (G->cap2) { cudaStreamDestroy(G->cap2); G->cap2 = nullptr; }
    for (void* q : G->allocs) cudaFree(q);
    G->allocs.clear();
    for (gsstv_handle* x : G->h) gsstv_destroy(x);
    G->h.clear();
}

// Numbers the CTAs of one stage across the slabs' launches.
void number_stage(std::vector<SlabPart>& parts, const std::vector<int>& grids) {
    int base = 0, total = 0;
    for (int g : grids) total += g;
    for (size_t s = 0; s < parts.size(); ++s) {
        parts[s].cta_base = base;
        parts[s].cta_total = total;
        base += grids[s];
    }
}

// One pass from parity `par` on `st`: every stage on every slab, then the halos.
int slabs_enqueue(gsstv_slabs* G, int par, cudaStream_t st, bool in_graph = false) {
    const int S = G->S;
    const IterParams ip = iparams(G->h[0], par);
    for (int s = 0; s < S; ++s) {
        gsstv_handle* x = G->h[s];
        TRY(map_launch(launch_k1_tma(GSSTV_FP32, x->g, x->maps[par], bufs(x, par), ip, G->sc, G->l1,
                                     G->k1_chunk[s], G->k1p[s], st)));
    }
    auto k1_finish = [&](int gated, cudaGraphConditionalHandle cond) -> int {
        return map_launch(launch_search_finish(2, G->sc, G->l1, 2, G->l1.k1_n, G->l1.k1_s, G->k1p[0].cta_total, st,
                                               gated, cond));
    };
    auto search = [&](cudaStream_t q) -> int {
        for (int s = 0; s < S; ++s) {
            gsstv_handle* x = G->h[s];
            TRY(map_launch(launch_window(GSSTV_FP32, x->g, bufs(x, par), ip, G->sc, G->l1, G->win_cap, G->winp[s],
                                         q)));
        }
        TRY(map_launch(launch_search_finish(0, G->sc, G->l1, 2, G->l1.k1_n, G->l1.k1_s, G->winp[0].cta_total, q)));
        for (int level = 0; level < 3; ++level)
            for (int s = 0; s < S; ++s) {
                gsstv_handle* x = G->h[s];
                TRY(map_launch(launch_fallback(GSSTV_FP32, level, x->g, bufs(x, par), ip, G->sc, G->l1, G->radp[s],
                                               q)));
            }
        for (int s = 0; s < S; ++s) {
            gsstv_handle* x = G->h[s];
            TRY(map_launch(launch_gather(GSSTV_FP32, x->g, bufs(x, par), ip, G->sc, G->l1, G->gatp[s], q)));
        }
        TRY(map_launch(launch_search_finish(1, G->sc, G->l1, 2, nullptr, nullptr, 0, q)));
        return GSSTV_OK;
    };
    if (in_graph) {
        TRY(capture_if_search(st, G->cap2, [&](cudaGraphConditionalHandle c) { return k1_finish(1, c); }, search));
    } else {
        TRY(k1_finish(0, 0));
        TRY(search(st));
    }
    for (int s = 0; s < S; ++s) {
        gsstv_handle* x = G->h[s];
        TRY(map_launch(launch_k2(GSSTV_FP32, x->g, bufs(x, par), ip, G->sc, G->k2_part, G->k2_cap, G->k2p[s], st)));
    }
    // halo exchange into the buffers the next pass reads (parity par ^ 1)
    const int nx = par ^ 1;
    for (int s = 0; s + 1 < S; ++s) {
        gsstv_handle* lo = G->h[s];
        gsstv_handle* hi = G->h[s + 1];
        const size_t plane = (size_t)lo->g.n1 * lo->g.p2 * sizeof(float);
        const size_t cube_lo = (size_t)lo->g.cube * sizeof(float), cube_hi = (size_t)hi->g.cube * sizeof(float);
        // the band above slab s (its top halo) is slab s+1's first owned band
        const size_t dst_top = (size_t)(G->B1[s] - G->L0[s]) * plane;
        const size_t src_top = (size_t)(G->B1[s] - G->L0[s + 1]) * plane;
        struct Pl { void* d; const void* s; int n; };
        const Pl top[4] = {{lo->u[nx], hi->u[nx], 1}, {lo->q[nx], hi->q[nx], 1},
                           {lo->y1[nx], hi->y1[nx], 2}, {lo->y2[nx], hi->y2[nx], 2}};
        for (const Pl& q : top)
            TRY(cuda_rc(cudaMemcpy2DAsync((char*)q.d + dst_top, cube_lo, (const char*)q.s + src_top, cube_hi, plane,
                                          (size_t)q.n, cudaMemcpyDeviceToDevice, st)));
        // the band below slab s+1 (its bottom halo) is slab s's last owned band
        const size_t dst_bot = (size_t)(G->B1[s] - 1 - G->L0[s + 1]) * plane;
        const size_t src_bot = (size_t)(G->B1[s] - 1 - G->L0[s]) * plane;
        TRY(cuda_rc(cudaMemcpy2DAsync((char*)hi->y2[nx] + dst_bot, cube_hi, (const char*)lo->y2[nx] + src_bot, cube_lo,
                                      plane, 2, cudaMemcpyDeviceToDevice, st)));
    }
    return GSSTV_OK;
}

int slabs_build_graph(gsstv_slabs* G, int par, int len) {
    cudaGraph_t graph = nullptr;
    TRY(cuda_rc(cudaStreamBeginCapture(G->cap, cudaStreamCaptureModeThreadLocal)));
    int rc = GSSTV_OK;
    int q = par;
    for (int k = 0; k < len && rc == GSSTV_OK; ++k) {
        rc = slabs_enqueue(G, q, G->cap, true);
        q ^= 1;
    }
    cudaError_t e = cudaStreamEndCapture(G->cap, &graph);
    if (rc != GSSTV_OK) { if (graph) cudaGraphDestroy(graph); return rc; }
    if (e != cudaSuccess) return GSSTV_ERR_CUDA;
    e = cudaGraphInstantiate(&G->gexec[par], graph, 0);
    cudaGraphDestroy(graph);
    return cuda_rc(e);
}

int slabs_run(gsstv_slabs* G, int n) {
    const int Gl = G->p.graph_iters > 0 ? ((G->p.graph_iters + 1) / 2) * 2 : 0;
    while (n > 0) {
        if (Gl > 0 && n >= Gl) {
            if (G->graph_len != Gl) {
                for (int k = 0; k < 2; ++k)
                    if (G->gexec[k]) { cudaGraphExecDestroy(G->gexec[k]); G->gexec[k] = nullptr; }
            }
            if (!G->gexec[G->parity]) TRY(slabs_build_graph(G, G->parity, Gl));
            G->graph_len = Gl;
            TRY(cuda_rc(cudaGraphLaunch(G->gexec[G->parity], G->st)));
            n -= Gl;
            G->stats.iterations += Gl;
        } else {
            TRY(slabs_enqueue(G, G->parity, G->st));
            G->parity ^= 1;
            --n;
            G->stats.iterations += 1;
        }
    }
    return GSSTV_OK;
}

int slabs_read_scalars(gsstv_slabs* G, Scal* out) {
    TRY(cuda_rc(cudaMemcpyAsync(out, G->sc, sizeof(Scal), cudaMemcpyDeviceToHost, G->st)));
    return cuda_rc(cudaStreamSynchronize(G->st));
}

int slabs_upload_scalars(gsstv_slabs* G) {
    Scal s = initial_scalars(G->p);
    TRY(cuda_rc(cudaMemcpyAsync(G->sc, &s, sizeof(Scal), cudaMemcpyHostToDevice, G->st)));
    return cuda_rc(cudaStreamSynchronize(G->st));
}

// float32 copies between a whole-cube dense view (ncubes cubes of N floats)
// and the stored bands [b0, b1) of one slab (pitched, its own cube stride)
int slab_copy(gsstv_slabs* G, int s, const float* view, void* store, int ncubes, int b0, int b1, bool to_store,
              const double* scale) {
    gsstv_handle* x = G->h[s];
    const long long N = (long long)G->n1 * G->n2 * G->n3;
    const long long dense_off = (long long)b0 * G->n1 * G->n2;
    const long long store_off = (long long)(b0 - G->L0[s]) * G->n1 * x->g.p2;
    float* st_ = (float*)store + store_off;
    if (to_store)
        return map_launch(launch_copy_f32(view + dense_off, G->n2, N, st_, x->g.p2, x->g.cube, G->n1, G->n2,
                                          b1 - b0, ncubes, nullptr, G->st));
    return map_launch(launch_copy_f32(st_, x->g.p2, x->g.cube, const_cast<float*>(view) + dense_off, G->n2, N,
                                      G->n1, G->n2, b1 - b0, ncubes, scale, G->st));
}

}  // namespace

int gsstv_slabs_destroy(gsstv_slabs* G) {
    if (!G) return GSSTV_OK;
    slabs_free(G);
    delete G;
    return GSSTV_OK;
}

int gsstv_slabs_create(gsstv_slabs** out, int n1, int n2, int n3, int nslabs, const gsstv_params* p, void* stream) {
    if (!out) return GSSTV_ERR_ARG;
    *out = nullptr;
    if (!shape_ok(n1, n2, n3) || nslabs < 1 || nslabs > n3) return GSSTV_ERR_ARG;
    TRY(check_params(p));
    if (p->storage != GSSTV_FP32) return GSSTV_ERR_ARG;
    gsstv_slabs* G = new gsstv_slabs();
    G->n1 = n1; G->n2 = n2; G->n3 = n3; G->S = nslabs;
    G->p = *p;
    G->st = (cudaStream_t)stream;
    int rc = GSSTV_OK;
    for (int s = 0; s < nslabs && rc == GSSTV_OK; ++s) {
        const int b0 = (int)((long long)s * n3 / nslabs), b1 = (int)((long long)(s + 1) * n3 / nslabs);
        const int l0 = std::max(b0 - 1, 0), l1 = std::min(b1 + 1, n3);
        G->B0.push_back(b0); G->B1.push_back(b1); G->L0.push_back(l0);
        gsstv_handle* x = nullptr;
        rc = gsstv_create(&x, n1, n2, l1 - l0, p, stream);
        if (rc == GSSTV_OK && x->k1_variant != 1) rc = GSSTV_ERR_ARG;    // the split runs the TMA-fed K1
        if (x) G->h.push_back(x);
        if (rc == GSSTV_OK) {
            SlabPart sp;
            sp.band0 = l0; sp.n3g = n3; sp.o0 = b0 - l0; sp.o1 = b1 - l0;
            G->k1p.push_back(sp); G->winp.push_back(sp); G->radp.push_back(sp);
            G->gatp.push_back(sp); G->k2p.push_back(sp);
        }
    }
    if (rc == GSSTV_OK && cudaStreamCreateWithFlags(&G->cap, cudaStreamNonBlocking) != cudaSuccess) {
        G->cap = nullptr;
        rc = GSSTV_ERR_CUDA;
    }
    if (rc == GSSTV_OK && cudaStreamCreateWithFlags(&G->cap2, cudaStreamNonBlocking) != cudaSuccess) {
        G->cap2 = nullptr;
        rc = GSSTV_ERR_CUDA;
    }
    if (rc == GSSTV_OK) {
        // each stage's launches, numbered across the slabs
        std::vector<int> gk1, gw, gr, gg, gk2;
        int max_chunk = 0;
        for (int s = 0; s < nslabs; ++s) {
            const Geom& g = G->h[s]->g;
            const int c = k1_tma_part_chunk(g, G->k1p[s], 0);
            G->k1_chunk.push_back(c);
            max_chunk = std::max(max_chunk, c);
            gk1.push_back(k1_tma_grid(g, G->k1p[s], c));
            gw.push_back(window_grid(g, G->winp[s], 1 << 30));
            gr.push_back(radix_grid(g, G->radp[s]));
            gg.push_back(gather_grid(g, G->gatp[s]));
            gk2.push_back(k2_grid(g, G->k2p[s], 1 << 30));
        }
        for (auto& sp : G->k1p) sp.max_chunk = max_chunk;
        number_stage(G->k1p, gk1);
        number_stage(G->winp, gw);
        number_stage(G->radp, gr);
        number_stage(G->gatp, gg);
        number_stage(G->k2p, gk2);
        const long long k1_total = G->k1p[0].cta_total, w_total = G->winp[0].cta_total;
        G->win_cap = 1 << 30;
        G->k2_cap = 1 << 30;
        const size_t part_n = (size_t)std::max(4 * k1_total, 2 * w_total);
        rc = slabs_alloc(G, (void**)&G->sc, sizeof(Scal));
        if (rc == GSSTV_OK) rc = slabs_alloc(G, (void**)&G->l1.cand[0], kCandCap * sizeof(float));
        if (rc == GSSTV_OK) rc = slabs_alloc(G, (void**)&G->l1.cand[1], kCandCap * sizeof(float));
        if (rc == GSSTV_OK) rc = slabs_alloc(G, (void**)&G->l1.hcnt, 2 * kHistBins * sizeof(unsigned long long));
        if (rc == GSSTV_OK) rc = slabs_alloc(G, (void**)&G->l1.hres, 2 * kHistBins * sizeof(unsigned long long));
        if (rc == GSSTV_OK) rc = slabs_alloc(G, (void**)&G->l1.k1_n, part_n * sizeof(unsigned long long));
        if (rc == GSSTV_OK) rc = slabs_alloc(G, (void**)&G->l1.k1_s, part_n * sizeof(double));
        if (rc == GSSTV_OK) rc = slabs_alloc(G, (void**)&G->l1.khist, 2 * (size_t)kK1Bins * sizeof(unsigned));
        if (rc == GSSTV_OK) rc = slabs_alloc(G, (void**)&G->l1.nh, 2 * 3 * (size_t)kNarrowBins * sizeof(unsigned));
        if (rc == GSSTV_OK) rc = slabs_alloc(G, (void**)&G->l1.nbinned, 2 * sizeof(unsigned));
        if (rc == GSSTV_OK)
            rc = slabs_alloc(G, (void**)&G->k2_part, 3 * (size_t)G->k2p[0].cta_total * sizeof(double));
    }
    if (rc == GSSTV_OK) rc = slabs_upload_scalars(G);
    if (rc != GSSTV_OK) {
        slabs_free(G);
        delete G;
        return rc;
    }
    *out = G;
    return GSSTV_OK;
}

int gsstv_slabs_load_observation(gsstv_slabs* G, const float* d_v) {
    if (!G || !d_v) return GSSTV_ERR_ARG;
    for (int s = 0; s < G->S; ++s) {
        gsstv_handle* x = G->h[s];
        const Geom& g = x->g;
        const float* src = d_v + (size_t)G->L0[s] * G->n1 * G->n2;
        TRY(cuda_rc(cudaMemcpy2DAsync(x->v, (size_t)g.p2 * 4, src, (size_t)g.n2 * 4, (size_t)g.n2 * 4,
                                      (size_t)g.n3 * g.n1, cudaMemcpyDeviceToDevice, G->st)));
    }
    return GSSTV_OK;
}

int gsstv_slabs_reset_state(gsstv_slabs* G) {
    if (!G) return GSSTV_ERR_ARG;
    TRY(cuda_rc(cudaStreamSynchronize(G->st)));
    for (gsstv_handle* x : G->h) TRY(gsstv_reset_state(x));
    G->parity = 0;
    return slabs_upload_scalars(G);
}

int gsstv_slabs_iterate(gsstv_slabs* G, int n, int* iters_done) {
    if (!G || n < 0) return GSSTV_ERR_ARG;
    if (iters_done) *iters_done = 0;
    int done = 0;
    Scal s;
    if (G->p.tol > 0.0) {
        while (done < n) {
            const int blk = std::min(G->p.check_every, n - done);
            TRY(slabs_run(G, blk));
            done += blk;
            TRY(slabs_read_scalars(G, &s));
            TRY(error_of(s));
            G->stats.last_rel_change = s.u2 > 0 ? std::sqrt(s.du2 / s.u2) : INFINITY;
            if (s.u2 > 0 && std::sqrt(s.du2 / s.u2) < G->p.tol) break;
        }
    } else {
        TRY(slabs_run(G, n));
        done = n;
        TRY(slabs_read_scalars(G, &s));
        TRY(error_of(s));
        G->stats.last_rel_change = s.u2 > 0 ? std::sqrt(s.du2 / s.u2) : INFINITY;
    }
    for (gsstv_handle* x : G->h) x->parity = G->parity;
    G->stats.last_tau_s = s.ctl[0].tau;
    G->stats.last_tau_t = s.ctl[1].tau;
    G->stats.last_l2_scale = s.c[G->parity];
    G->stats.tau_window_hits = s.ctl[0].hits + s.ctl[1].hits;
    G->stats.tau_exact_runs = s.ctl[0].exact_runs + s.ctl[1].exact_runs;
    G->stats.tau_retry_hits = s.ctl[0].retry_hits + s.ctl[1].retry_hits;
    G->stats.search_passes = s.gate_opens;
    if (iters_done) *iters_done = done;
    return GSSTV_OK;
}

int gsstv_slabs_get_state(gsstv_slabs* G, const gsstv_state_view* v) {
    if (!G || !view_ok(v)) return GSSTV_ERR_ARG;
    const int par = G->parity;
    for (int s = 0; s < G->S; ++s) {
        gsstv_handle* x = G->h[s];
        const int b0 = G->B0[s], b1 = G->B1[s];
        TRY(slab_copy(G, s, v->u, x->u[par], 1, b0, b1, false, nullptr));
        TRY(slab_copy(G, s, v->s, x->s[par], 1, b0, b1, false, nullptr));
        TRY(slab_copy(G, s, v->t, x->t[par], 1, b0, b1, false, nullptr));
        TRY(slab_copy(G, s, v->w1, x->w1[par], 6, b0, b1, false, nullptr));
        TRY(slab_copy(G, s, v->w2, x->w2[par], 6, b0, b1, false, nullptr));
        TRY(slab_copy(G, s, v->y1, x->y1[par], 2, b0, b1, false, nullptr));
        TRY(slab_copy(G, s, v->y2, x->y2[par], 2, b0, b1, false, nullptr));
        TRY(slab_copy(G, s, v->y3, x->y3[par], 1, b0, b1, false, nullptr));
        TRY(slab_copy(G, s, v->y4, x->q[par], 1, b0, b1, false, &G->sc->c[par]));
    }
    return cuda_rc(cudaStreamSynchronize(G->st));
}

int gsstv_slabs_set_state(gsstv_slabs* G, const gsstv_state_view* v) {
    if (!G || !view_ok(v)) return GSSTV_ERR_ARG;
    const int par = G->parity;
    for (int s = 0; s < G->S; ++s) {
        gsstv_handle* x = G->h[s];
        // the stored bands, halos included
        const int b0 = G->L0[s], b1 = G->L0[s] + x->g.n3;
        TRY(slab_copy(G, s, v->u, x->u[par], 1, b0, b1, true, nullptr));
        TRY(slab_copy(G, s, v->s, x->s[par], 1, b0, b1, true, nullptr));
        TRY(slab_copy(G, s, v->t, x->t[par], 1, b0, b1, true, nullptr));
        TRY(slab_copy(G, s, v->w1, x->w1[par], 6, b0, b1, true, nullptr));
        TRY(slab_copy(G, s, v->w2, x->w2[par], 6, b0, b1, true, nullptr));
        TRY(slab_copy(G, s, v->y1, x->y1[par], 2, b0, b1, true, nullptr));
        TRY(slab_copy(G, s, v->y2, x->y2[par], 2, b0, b1, true, nullptr));
        TRY(slab_copy(G, s, v->y3, x->y3[par], 1, b0, b1, true, nullptr));
        TRY(slab_copy(G, s, v->y4, x->q[par], 1, b0, b1, true, nullptr));
    }
    // y4 is now stored unscaled (c = 0); the threshold search starts afresh
    return slabs_upload_scalars(G);
}

int gsstv_slabs_solve(gsstv_slabs* G, const float* d_v, float* d_u, float* d_s, float* d_t, int* iters_done) {
    if (!G || !d_v || !d_u) return GSSTV_ERR_ARG;
    TRY(gsstv_slabs_load_observation(G, d_v));
    TRY(gsstv_slabs_reset_state(G));
    TRY(gsstv_slabs_iterate(G, G->p.max_iter, iters_done));
    const int par = G->parity;
    for (int s = 0; s < G->S; ++s) {
        gsstv_handle* x = G->h[s];
        TRY(slab_copy(G, s, d_u, x->u[par], 1, G->B0[s], G->B1[s], false, nullptr));
        if (d_s) TRY(slab_copy(G, s, d_s, x->s[par], 1, G->B0[s], G->B1[s], false, nullptr));
        if (d_t) TRY(slab_copy(G, s, d_t, x->t[par], 1, G->B0[s], G->B1[s], false, nullptr));
    }
    return cuda_rc(cudaStreamSynchronize(G->st));
}

int gsstv_slabs_get_stats(gsstv_slabs* G, gsstv_stats* out) {
    if (!G || !out) return GSSTV_ERR_ARG;
    *out = G->stats;
    return GSSTV_OK;
}

int gsstv_slabs_count(const gsstv_slabs* G, int* bands_out) {
    if (!G) return 0;
    if (bands_out)
        for (int s = 0; s < G->S; ++s) bands_out[s] = G->B1[s] - G->B0[s];
    return G->S;
}

const char* gsstv_strerror(int code) {
    switch (code) {
        case GSSTV_OK: return "ok";
        case GSSTV_ERR_ARG: return "invalid argument";
        case GSSTV_ERR_OOM: return "device allocation failed";
        case GSSTV_ERR_CUDA: return "CUDA call failed";
        case GSSTV_ERR_NONFINITE: return "non-finite value in the l2-ball norm";
        case GSSTV_ERR_TIMEOUT: return "bounded device wait timed out";
        case GSSTV_ERR_INTERNAL: return "internal consistency check failed";
    }
    return "unknown error code";
}

}  // extern "C"
