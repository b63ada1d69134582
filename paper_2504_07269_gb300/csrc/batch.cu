// Batched solve of many independent space-time problems of uneven size (spatial mesh, n_t,
// temporal degree) in the mixed precision of st_fdm_solve: FP64 flexible GMRES on each problem's
// Kronecker system (eq. LGS), right-preconditioned by its complex-FP32 fast-diagonalisation solve
// (Section 3, steps 2-4), all problems advancing together.
//
//   * a plan (st_batch_create) packs the problems' space-time vectors, builds the block tables of
//     the grouped kernels and a work list of all (problem, shift) spatial systems sorted by cost
//     (largest first), and sizes the GMRES basis from free memory;
//   * a project-written autotuner times the candidate tile shapes of the grouped transforms and
//     the CTAs per SM of the persistent factor-and-solve on this plan's data and keeps the
//     fastest, cached per shape signature for the process;
//   * a whole restart cycle -- the residual, the restart test, m Arnoldi steps (transforms,
//     persistent factor-and-solve launch, operator apply, two Gram-Schmidt passes, rotations)
//     and the solution update -- is launched with no host decision inside it, so it is captured
//     once in a CUDA graph and replayed; the host reads one counter per cycle.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "device.cuh"
#include "plan_rules.h"

namespace stfdm {

int kb_seg_blocks(long long n);
int kb_res_blocks(int n_t, int n_x);
int kb_max_vectors();
int kb_xform_shapes();
void kb_xform_shape(int s, int* bm, int* bn);
cudaError_t kb_launch_xform(int shape, int ntiles, const BatchProb* probs, const int* tile0, int P, const int* on,
                            int which, const void* in, bool in_c128, float2* out, cudaStream_t st);
cudaError_t kb_launch_residual(int nblocks, const BatchProb* probs, const int* blk0, int P, const int* off,
                               double* partials, double2* w, double* rr, double* ff, cudaStream_t st);
cudaError_t kb_launch_apply(int nblocks, const BatchProb* probs, const int* blk0, int P, const int* on, const float2* Z,
                            double2* w, cudaStream_t st);
cudaError_t kb_launch_multidot(int nseg, const BatchProb* probs, const int* seg0, int P, const int* on,
                               const double2* Vb, size_t vs, int nv, const double2* w, double2* partial, double2* out,
                               int out_stride, cudaStream_t st);
cudaError_t kb_launch_multiaxpy(int nseg, const BatchProb* probs, const int* seg0, int P, const int* on,
                                const double2* Vb, size_t vs, int nv, const double2* c, int c_stride, double2* w,
                                cudaStream_t st);
cudaError_t kb_launch_scale(int nseg, const BatchProb* probs, const int* seg0, int P, const int* on, const double* inv,
                            const double2* w, double2* out, cudaStream_t st);
cudaError_t kb_launch_update_x(int nseg, const BatchProb* probs, const int* seg0, int P, const int* jdone,
                               const float2* Z, size_t zs, const double2* y, int m, cudaStream_t st);
cudaError_t kb_launch_init(const BatchGm& gm, int P, int m, cudaStream_t st);
cudaError_t kb_launch_cycle_start(const BatchGm& gm, int P, int m, double tol, int maxit, cudaStream_t st);
cudaError_t kb_launch_arnoldi(const BatchGm& gm, int P, int m, int j, double tol, int maxit, cudaStream_t st);
cudaError_t kb_launch_solve_y(const BatchGm& gm, int P, int m, cudaStream_t st);
cudaError_t kb_launch_mark_factored(const BatchBand* probs, const int* active, int* factored, int P, cudaStream_t st);
cudaError_t launch_stencil_A(const SpaceMats& sm, const void* in, bool in_c64, const double2* add, double sign,
                             double2* out, cudaStream_t st);
cudaError_t launch_add_row(int n_t, int n_x, void* psi, const void* psi0, bool c64, cudaStream_t st);

}  // namespace stfdm

using namespace stfdm;

namespace {

#define BT_TRY(expr)                                                                         \
    do {                                                                                     \
        cudaError_t _e = (expr);                                                             \
        if (_e != cudaSuccess)                                                               \
            return fail(ST_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e));    \
    } while (0)

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int dev) {
        cudaGetDevice(&prev);
        if (dev >= 0 && dev != prev) cudaSetDevice(dev);
    }
    ~DevGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// tuned choices, per shape signature, for the life of the process
struct TuneChoice {
    int xform_shape = 0;
    int ctas_per_sm = 2;
};
std::mutex g_tune_mutex;
std::map<std::string, TuneChoice> g_tune_cache;

constexpr int BATCH_MAX_RESTART = 20;
constexpr int BATCH_MIN_RESTART = 4;    // shortest basis chosen to make room for kept factors

}  // namespace

struct st_batch {
    int device = 0;
    int P = 0;
    int sm_count = 0;
    std::vector<st_fdm*> hs;
    std::vector<long long> off;
    long long N = 0;          // packed space-time length
    long long spatial = 0;    // packed spatial length (A_x psi0)
    int m = 0;                // restart length
    double tol = 1e-12;
    int maxit = 40;
    int use_graph = 1;
    int b_max = 0;
    int n_items = 0;
    int n_res = 0, n_seg = 0;
    std::vector<int> ntiles;  // per transform shape
    TuneChoice choice;
    int tuned = 0;
    double tune_seconds = 0;
    int grid = 0;
    size_t L_stride = 0, D_stride = 0;
    size_t bytes = 0;
    int cycles = 0;
    // host mirrors
    std::vector<BatchProb> hprob;
    std::vector<std::vector<int>> htile0;
    // device
    cudaStream_t cs = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    BatchProb* d_prob = nullptr;
    BatchBand* d_band = nullptr;
    int2* d_items = nullptr;
    int* d_res0 = nullptr;
    int* d_seg0 = nullptr;
    int* d_tile0 = nullptr;   // all shapes, concatenated (P + 1 each)
    double2* V = nullptr;     // (m + 1) x N
    float2* Z = nullptr;      // m x N
    double2* w = nullptr;     // N
    float2* G = nullptr;      // N
    double2* apsi0 = nullptr; // spatial
    double* res_part = nullptr;
    double2* dot_part = nullptr;
    float2* win = nullptr;
    float2* Lslots = nullptr;
    float2* Dslots = nullptr;
    int* counter = nullptr;
    int* factored = nullptr;  // per problem: kept factors stored (set after its first application)
    int2* d_kitems = nullptr; // work list of the kept-factor systems
    int n_kitems = 0;
    int kept = 0;             // problems with kept factors
    int kb_max = 0;           // widest band among them
    size_t kept_bytes = 0;
    std::vector<BatchBand> hband;
    int* status = nullptr;
    void* gm_mem = nullptr;
    BatchGm gm{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t graph_nodes = 0;
    std::vector<void*> allocs;
};

namespace {

st_status balloc(st_batch* b, void** p, size_t bytes, const char* what) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? ST_ERR_OOM : ST_ERR_CUDA,
                    std::string("st_batch: cudaMalloc(") + what + ", " + std::to_string(bytes) + " B): " +
                        cudaGetErrorString(e));
    }
    b->allocs.push_back(*p);
    b->bytes += bytes;
    return ST_OK;
}

void destroy(st_batch* b) {
    if (!b) return;
    DevGuard g(b->device);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (void* p : b->allocs) cudaFree(p);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->cs) cudaStreamDestroy(b->cs);
    delete b;
}

const int* tile0_of(const st_batch* b, int shape) { return b->d_tile0 + (size_t)shape * (b->P + 1); }

// one restart cycle of every problem: no host decision, so it can be captured in a graph
cudaError_t enqueue_cycle(st_batch* b, cudaStream_t st) {
    const int P = b->P, m = b->m, MV = kb_max_vectors();
    const size_t N = (size_t)b->N;
    const BatchGm& gm = b->gm;
    const int shape = b->choice.xform_shape;
    cudaError_t e;
#define BQ(x)                             \
    do {                                  \
        e = (x);                          \
        if (e != cudaSuccess) return e;   \
    } while (0)
    BQ(cudaMemsetAsync(gm.pending, 0, sizeof(int), st));
    BQ(kb_launch_residual(b->n_res, b->d_prob, b->d_res0, P, gm.stopped, b->res_part, b->w, gm.rr, gm.ff, st));
    BQ(kb_launch_cycle_start(gm, P, m, b->tol, b->maxit, st));
    BQ(kb_launch_scale(b->n_seg, b->d_prob, b->d_seg0, P, gm.active, gm.inv, b->w, b->V, st));
    for (int j = 0; j < m; ++j) {
        double2* Vj = b->V + (size_t)j * N;
        float2* Zj = b->Z + (size_t)j * N;
        BQ(kb_launch_xform(shape, b->ntiles[shape], b->d_prob, tile0_of(b, shape), P, gm.active, 0, Vj, true, b->G, st));
        BQ(band_batch_launch(b->d_band, b->d_items, b->n_items, gm.active, b->factored, b->counter, b->b_max, b->win,
                             b->Lslots, b->L_stride, b->Dslots, b->D_stride, b->status, b->grid, st));
        if (b->n_kitems > 0) {
            // systems whose factors are kept from an earlier application: substitutions only
            BQ(subst_batch_launch(b->d_band, b->d_kitems, b->n_kitems, gm.active, b->factored, b->kb_max, b->status,
                                  true, st));
            BQ(subst_batch_launch(b->d_band, b->d_kitems, b->n_kitems, gm.active, b->factored, b->kb_max, b->status,
                                  false, st));
            BQ(kb_launch_mark_factored(b->d_band, gm.active, b->factored, P, st));
        }
        BQ(kb_launch_xform(shape, b->ntiles[shape], b->d_prob, tile0_of(b, shape), P, gm.active, 1, b->G, false, Zj, st));
        BQ(kb_launch_apply(b->n_res, b->d_prob, b->d_res0, P, gm.active, Zj, b->w, st));
        for (int pass = 0; pass < 2; ++pass) {
            BQ(kb_launch_multidot(b->n_seg, b->d_prob, b->d_seg0, P, gm.active, b->V, N, j + 1, b->w, b->dot_part,
                                  gm.h + pass * MV, 3 * MV, st));
            BQ(kb_launch_multiaxpy(b->n_seg, b->d_prob, b->d_seg0, P, gm.active, b->V, N, j + 1, gm.h + pass * MV,
                                   3 * MV, b->w, st));
        }
        BQ(kb_launch_multidot(b->n_seg, b->d_prob, b->d_seg0, P, gm.active, b->w, 0, 1, b->w, b->dot_part,
                              gm.h + 2 * MV, 3 * MV, st));
        BQ(kb_launch_arnoldi(gm, P, m, j, b->tol, b->maxit, st));
        if (j + 1 < m)
            BQ(kb_launch_scale(b->n_seg, b->d_prob, b->d_seg0, P, gm.active, gm.inv, b->w, b->V + (size_t)(j + 1) * N,
                               st));
    }
    BQ(kb_launch_solve_y(gm, P, m, st));
    BQ(kb_launch_update_x(b->n_seg, b->d_prob, b->d_seg0, P, gm.jdone, b->Z, N, gm.y, m, st));
#undef BQ
    return cudaSuccess;
}

std::string signature(const st_batch* b) {
    std::string s = "sm" + std::to_string(b->sm_count) + "|P" + std::to_string(b->P) + "|items" +
                    std::to_string(b->n_items) + "|bmax" + std::to_string(b->b_max);
    for (const BatchProb& p : b->hprob) s += "|" + std::to_string(p.n_t) + "x" + std::to_string(p.n_x);
    return s;
}

// time `fn` once after one untimed run (milliseconds)
template <typename Fn>
st_status time_ms(cudaStream_t st, Fn fn, float* ms) {
    cudaEvent_t a, c;
    BT_TRY(cudaEventCreate(&a));
    BT_TRY(cudaEventCreate(&c));
    cudaError_t e = fn();
    if (e == cudaSuccess) e = cudaEventRecord(a, st);
    if (e == cudaSuccess) e = fn();
    if (e == cudaSuccess) e = cudaEventRecord(c, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(c);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, c);
    cudaEventDestroy(a);
    cudaEventDestroy(c);
    if (e != cudaSuccess) return fail(ST_ERR_CUDA, std::string("st_batch tuner: ") + cudaGetErrorString(e));
    return ST_OK;
}

// Autotuner: every transform tile shape on one forward transform of the whole batch, and 1 or 2
// CTAs per SM for the persistent factor-and-solve on the costliest items (work list prefix).
st_status tune(st_batch* b) {
    const auto t0 = std::chrono::steady_clock::now();
    const std::string key = signature(b);
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            b->choice = it->second;
            b->tuned = 2;
            return ST_OK;
        }
    }
    cudaStream_t st = b->cs;
    const int P = b->P;
    std::vector<int> ones(P, 1);
    BT_TRY(cudaMemcpyAsync(b->gm.active, ones.data(), P * sizeof(int), cudaMemcpyHostToDevice, st));
    BT_TRY(cudaMemsetAsync(b->V, 0, (size_t)b->N * sizeof(double2), st));
    BT_TRY(cudaStreamSynchronize(st));
    TuneChoice best;
    float best_ms = 1e30f;
    for (int s = 0; s < kb_xform_shapes(); ++s) {
        float ms = 0;
        st_status r = time_ms(st, [&]() {
            return kb_launch_xform(s, b->ntiles[s], b->d_prob, tile0_of(b, s), P, b->gm.active, 0, b->V, true, b->G, st);
        }, &ms);
        if (r != ST_OK) return r;
        if (ms < best_ms) {
            best_ms = ms;
            best.xform_shape = s;
        }
    }
    // the costliest items: three full waves at two CTAs per SM
    const int occ = std::min(2, band_batch_occupancy(b->b_max));
    if (occ < 1) return fail(ST_ERR_UNSUPPORTED, "st_batch: the factor kernel does not fit on an SM");
    best.ctas_per_sm = occ;
    if (occ == 2) {
        const int sample = std::min(b->n_items, 3 * 2 * b->sm_count);
        BT_TRY(cudaMemsetAsync(b->G, 0, (size_t)b->N * sizeof(float2), st));
        float tms[3] = {0, 0, 0};
        for (int c = 1; c <= 2; ++c) {
            st_status r = time_ms(st, [&]() {
                return band_batch_launch(b->d_band, b->d_items, sample, b->gm.active, nullptr, b->counter, b->b_max, b->win,
                                         b->Lslots, b->L_stride, b->Dslots, b->D_stride, b->status, c * b->sm_count, st);
            }, &tms[c]);
            if (r != ST_OK) return r;
        }
        best.ctas_per_sm = (tms[1] < tms[2]) ? 1 : 2;
    }
    BT_TRY(cudaMemsetAsync(b->status, 0, 2 * sizeof(int), st));
    BT_TRY(cudaStreamSynchronize(st));
    b->choice = best;
    b->tuned = 1;
    b->tune_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = best;
    return ST_OK;
}

st_status build_graph(st_batch* b) {
    if (b->exec) return ST_OK;
    cudaStream_t st = b->cs;
    BT_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_cycle(b, st);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(st, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(ST_ERR_CUDA, std::string("st_batch: graph capture: ") +
                                     cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return fail(ST_ERR_CUDA, std::string("st_batch: graph instantiate: ") + cudaGetErrorString(e));
    }
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    b->graph = g;
    b->exec = ex;
    b->graph_nodes = nn;
    return ST_OK;
}

}  // namespace

// ==================================================================== ABI
extern "C" st_status st_batch_create(st_fdm* const* hs, int count, const st_batch_opts* opts, st_batch** out) {
    if (!out) return fail(ST_ERR_ARG, "st_batch_create: out is NULL");
    *out = nullptr;
    if (!hs || count < 1) return fail(ST_ERR_ARG, "st_batch_create: need at least one handle");
    for (int i = 0; i < count; ++i) {
        if (!hs[i]) return fail(ST_ERR_ARG, "st_batch_create: NULL handle");
        if (hs[i]->spatial != 0)
            return fail(ST_ERR_UNSUPPORTED, "st_batch_create: batched plans use the banded spatial solver (structured grids)");
    }
    const int dev = hs[0]->device;
    for (int i = 1; i < count; ++i)
        if (hs[i]->device != dev) return fail(ST_ERR_ARG, "st_batch_create: handles on different devices");
    st_batch_opts o;
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (o.tol < 0 || o.max_sweeps < 0 || o.restart < 0) return fail(ST_ERR_ARG, "st_batch_create: negative option");
    DevGuard guard(dev);
    st_batch* b = new (std::nothrow) st_batch();
    if (!b) return fail(ST_ERR_OOM, "st_batch_create: host allocation");
    b->device = dev;
    b->P = count;
    b->hs.assign(hs, hs + count);
    b->tol = o.tol > 0 ? o.tol : 1e-12;
    b->maxit = o.max_sweeps > 0 ? o.max_sweeps : 40;
    b->use_graph = o.no_graph ? 0 : 1;
    b->sm_count = hs[0]->sm_count;
    st_status s = ST_OK;
    auto bail = [&](st_status r) {
        destroy(b);
        return r;
    };
    if (cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(ST_ERR_CUDA, "st_batch_create: stream/event creation"));
    // packing, descriptors, block tables
    const int P = count;
    b->off.resize(P);
    std::vector<int> res0(P + 1), seg0(P + 1);
    std::vector<BatchBand> band(P);
    b->hprob.resize(P);
    long long N = 0, spatial = 0;
    size_t max_nb = 0, max_nx = 0;
    int b_max = 0;
    for (int p = 0; p < P; ++p) {
        const st_fdm* h = hs[p];
        const int n_t = h->tm.n_t, n_x = h->sm.n_x;
        BatchProb& pr = b->hprob[p];
        std::memset(&pr, 0, sizeof(pr));
        pr.n_t = n_t;
        pr.n_x = n_x;
        pr.m = h->sm.m;
        pr.tband = h->tm.p == 1 ? 3 : 5;
        pr.Mc = h->sm.Mc; pr.Mw = h->sm.Mw; pr.Ms = h->sm.Ms; pr.Md = h->sm.Md;
        pr.Ac = h->sm.Ac; pr.Aw = h->sm.Aw; pr.As = h->sm.As; pr.Ad = h->sm.Ad;
        pr.Mb = h->dt.Mb;
        pr.Bb = h->dt.Bb;
        pr.m_t = h->dt.m;
        pr.Y32 = h->xf32[XF_Y];
        pr.X32 = h->xf32[XF_X];
        pr.off = N;
        const long long np = (long long)n_t * n_x;
        pr.psc = std::ldexp(1.0, (int)std::lround(0.5 * std::log2((double)np)));
        b->off[p] = N;
        res0[p + 1] = res0[p] + kb_res_blocks(n_t, n_x);
        seg0[p + 1] = seg0[p] + kb_seg_blocks(np);
        N += np;
        spatial += n_x;
        const int bw = h->sm.m + 1;
        b_max = std::max(b_max, bw);
        max_nb = std::max(max_nb, (size_t)n_x * bw);
        max_nx = std::max(max_nx, (size_t)n_x);
        BatchBand& bb = band[p];
        std::memset(&bb, 0, sizeof(bb));
        bb.n = n_x;
        bb.m = h->sm.m;
        bb.b = bw;
        bb.Mc = (float)h->sm.Mc; bb.Mw = (float)h->sm.Mw; bb.Ms = (float)h->sm.Ms; bb.Md = (float)h->sm.Md;
        bb.Ac = (float)h->sm.Ac; bb.Aw = (float)h->sm.Aw; bb.As = (float)h->sm.As; bb.Ad = (float)h->sm.Ad;
        bb.shifts = h->s32;
    }
    if (res0[P] < 0 || seg0[P] < 0) return bail(fail(ST_ERR_UNSUPPORTED, "st_batch_create: batch too large"));
    b->N = N;
    b->spatial = spatial;
    b->b_max = b_max;
    b->n_res = res0[P];
    b->n_seg = seg0[P];
    if (band_batch_smem(b_max) > hs[0]->smem_optin)
        return bail(fail(ST_ERR_UNSUPPORTED, "st_batch_create: spatial band too wide for shared memory"));
    if (band_batch_prepare(b_max) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(ST_ERR_CUDA, "st_batch_create: factor kernel attributes"));
    }
    // work list: every (problem, shift), costliest (n_x b^2) first
    std::vector<int2> items;
    for (int p = 0; p < P; ++p)
        for (int k = 0; k < hs[p]->tm.n_t; ++k) items.push_back(make_int2(p, k));
    std::stable_sort(items.begin(), items.end(), [&](const int2& a, const int2& c) {
        const double ca = (double)band[a.x].n * band[a.x].b * band[a.x].b;
        const double cc = (double)band[c.x].n * band[c.x].b * band[c.x].b;
        return ca > cc;
    });
    b->n_items = (int)items.size();
    // transform tile tables for every candidate shape
    const int NS = kb_xform_shapes();
    std::vector<int> tile0((size_t)NS * (P + 1));
    b->ntiles.resize(NS);
    for (int sh = 0; sh < NS; ++sh) {
        int bm, bn;
        kb_xform_shape(sh, &bm, &bn);
        int* t = tile0.data() + (size_t)sh * (P + 1);
        t[0] = 0;
        for (int p = 0; p < P; ++p)
            t[p + 1] = t[p] + ((b->hprob[p].n_t + bm - 1) / bm) * ((b->hprob[p].n_x + bn - 1) / bn);
        b->ntiles[sh] = t[P];
    }
    // restart length: the basis holds m + 1 complex128 and m complex64 vectors (see below)
    const int occ = std::max(1, std::min(2, band_batch_occupancy(b_max)));
    b->grid = occ * b->sm_count;
    b->L_stride = max_nb;
    b->D_stride = max_nx;
    const size_t fixed = (size_t)N * (sizeof(double2) + sizeof(float2)) + (size_t)b->grid * max_nb * sizeof(float2) +
                         (size_t)b->grid * (size_t)(b_max + 32) * (b_max + 1) * sizeof(float2);
    int m = o.restart > 0 ? std::min(o.restart, BATCH_MAX_RESTART) : BATCH_MAX_RESTART;
    m = std::min(m, kb_max_vectors() - 1);
    if (o.restart <= 0) {
        // The FP32-preconditioned refinement converges within about ten applications whatever m is
        // (64-problem batch: 331 applications at m = 13, 330 at m = 4, and 19% less time at m = 4
        // with 18 instead of 9 problems kept), so the basis yields memory to the kept factors.
        size_t freeb = 0, total = 0;
        cudaMemGetInfo(&freeb, &total);
        const size_t avail = freeb > fixed ? freeb - fixed : 0;
        size_t factors = 0;
        if (!o.no_keep)
            for (int q = 0; q < P; ++q)
                if (band[q].b <= 256)
                    factors += ((size_t)b->hprob[q].n_t * band[q].n * ((size_t)band[q].b + 1) * sizeof(float2) + 255) / 256 * 256;
        m = batch_restart_for_factors((size_t)N, avail, factors, m, BATCH_MIN_RESTART);
    }
    b->m = m;
    // device buffers
    void* p;
#define BA(field, bytes, what)                                     \
    do {                                                           \
        s = balloc(b, &p, (bytes), what);                          \
        if (s != ST_OK) return bail(s);                            \
        b->field = reinterpret_cast<decltype(b->field)>(p);        \
    } while (0)
    BA(d_prob, sizeof(BatchProb) * P, "descriptors");
    BA(d_band, sizeof(BatchBand) * P, "band descriptors");
    BA(d_items, sizeof(int2) * items.size(), "work list");
    BA(d_res0, sizeof(int) * (P + 1), "residual table");
    BA(d_seg0, sizeof(int) * (P + 1), "segment table");
    BA(d_tile0, sizeof(int) * tile0.size(), "tile tables");
    BA(V, (size_t)(m + 1) * N * sizeof(double2), "GMRES basis");
    BA(Z, (size_t)m * N * sizeof(float2), "GMRES directions");
    BA(w, (size_t)N * sizeof(double2), "work vector");
    BA(G, (size_t)N * sizeof(float2), "FP32 transform buffer");
    BA(apsi0, (size_t)spatial * sizeof(double2), "A_x psi0");
    BA(res_part, (size_t)b->n_res * 2 * sizeof(double), "residual partials");
    BA(dot_part, (size_t)b->n_seg * kb_max_vectors() * sizeof(double2), "dot partials");
    BA(win, (size_t)b->grid * (b_max + 32) * (b_max + 1) * sizeof(float2), "factor windows");
    BA(Lslots, (size_t)b->grid * max_nb * sizeof(float2), "factor slots");
    BA(Dslots, (size_t)b->grid * max_nx * sizeof(float2), "pivot slots");
    BA(counter, sizeof(int), "work counter");
    BA(status, 2 * sizeof(int), "status");
    BA(factored, sizeof(int) * P, "factor flags");
#undef BA
    {
        // per-problem GMRES state, carved out of one allocation (every array 16-byte aligned);
        // the same walk runs twice: once to size the block, once to assign the pointers
        const int MV = kb_max_vectors();
        const size_t dP = P;
        auto layout = [&](char* base) {
            size_t at = 0;
            auto take = [&](size_t n) {
                char* r = base ? base + at : nullptr;
                at += (n + 15) / 16 * 16;
                return r;
            };
            BatchGm g{};
            g.H = reinterpret_cast<double2*>(take(dP * (m + 1) * m * sizeof(double2)));
            g.g = reinterpret_cast<double2*>(take(dP * (m + 1) * sizeof(double2)));
            g.sn = reinterpret_cast<double2*>(take(dP * m * sizeof(double2)));
            g.h = reinterpret_cast<double2*>(take(dP * 3 * MV * sizeof(double2)));
            g.y = reinterpret_cast<double2*>(take(dP * m * sizeof(double2)));
            g.cs = reinterpret_cast<double*>(take(dP * m * sizeof(double)));
            g.rr = reinterpret_cast<double*>(take(dP * sizeof(double)));
            g.ff = reinterpret_cast<double*>(take(dP * sizeof(double)));
            g.bnorm = reinterpret_cast<double*>(take(dP * sizeof(double)));
            g.rel = reinterpret_cast<double*>(take(dP * sizeof(double)));
            g.inv = reinterpret_cast<double*>(take(dP * sizeof(double)));
            g.hist = reinterpret_cast<double*>(take(dP * 16 * sizeof(double)));
            g.nh = reinterpret_cast<int*>(take(dP * sizeof(int)));
            g.its = reinterpret_cast<int*>(take(dP * sizeof(int)));
            g.stopped = reinterpret_cast<int*>(take(dP * sizeof(int)));
            g.active = reinterpret_cast<int*>(take(dP * sizeof(int)));
            g.jdone = reinterpret_cast<int*>(take(dP * sizeof(int)));
            g.pending = reinterpret_cast<int*>(take(sizeof(int)));
            if (base) b->gm = g;
            return at;
        };
        const size_t bytes = layout(nullptr);
        s = balloc(b, &b->gm_mem, bytes, "GMRES state");
        if (s != ST_OK) return bail(s);
        layout(static_cast<char*>(b->gm_mem));
    }
    for (int q = 0; q < P; ++q) band[q].rhs = b->G + b->off[q];
    // Kept factors: problems with the widest bands first (the factorisation costs n_x b^2 per system,
    // its storage n_x b), as long as they fit in the free memory left (less a reserve); their later
    // preconditioner applications only stream the factors (grouped substitutions, b <= 256).
    std::vector<int2> kitems;
    if (!o.no_keep) {
        size_t freeb = 0, total = 0;
        cudaMemGetInfo(&freeb, &total);
        const size_t reserve = (size_t)2 << 30;
        size_t budget = freeb > reserve ? (size_t)((freeb - reserve) * 0.9) : 0;
        std::vector<int> order(P);
        for (int q = 0; q < P; ++q) order[q] = q;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return band[x].b > band[y].b; });
        std::vector<size_t> loff(P, 0);
        size_t need = 0;
        std::vector<char> keep(P, 0);
        for (int q : order) {
            if (band[q].b > 256) continue;
            const size_t nt = (size_t)hs[q]->tm.n_t, nx = (size_t)band[q].n;
            // L then D; each problem's block 256-byte aligned (the bulk copies need 16-byte sources)
            const size_t bytes = (nt * nx * ((size_t)band[q].b + 1) * sizeof(float2) + 255) / 256 * 256;
            if (need + bytes > budget) continue;
            keep[q] = 1;
            loff[q] = need;
            need += bytes;
        }
        if (need > 0) {
            void* pk = nullptr;
            s = balloc(b, &pk, need, "kept factors");
            if (s == ST_OK) {
                float2* base = static_cast<float2*>(pk);
                for (int q = 0; q < P; ++q) {
                    if (!keep[q]) continue;
                    const size_t nt = (size_t)hs[q]->tm.n_t, nx = (size_t)band[q].n;
                    band[q].Lkeep = base + loff[q] / sizeof(float2);
                    band[q].Dkeep = band[q].Lkeep + nt * nx * band[q].b;
                    ++b->kept;
                    b->kb_max = std::max(b->kb_max, band[q].b);
                }
                b->kept_bytes = need;
                for (const int2& it : items)
                    if (keep[it.x]) kitems.push_back(it);
            } else {
                cudaGetLastError();   // not enough memory after all: refactorise everything
                s = ST_OK;
            }
        }
    }
    b->n_kitems = (int)kitems.size();
    if (b->n_kitems > 0) {
        void* pk = nullptr;
        s = balloc(b, &pk, sizeof(int2) * kitems.size(), "kept work list");
        if (s != ST_OK) return bail(s);
        b->d_kitems = static_cast<int2*>(pk);
    }
    b->hband = band;
    cudaStream_t st = b->cs;
    cudaError_t e = cudaMemcpyAsync(b->d_prob, b->hprob.data(), sizeof(BatchProb) * P, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_band, band.data(), sizeof(BatchBand) * P, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_res0, res0.data(), sizeof(int) * (P + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_seg0, seg0.data(), sizeof(int) * (P + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_tile0, tile0.data(), sizeof(int) * tile0.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && b->n_kitems > 0)
        e = cudaMemcpyAsync(b->d_kitems, kitems.data(), sizeof(int2) * kitems.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->factored, 0, sizeof(int) * P, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->status, 0, 2 * sizeof(int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return bail(fail(ST_ERR_CUDA, std::string("st_batch_create: upload: ") + cudaGetErrorString(e)));
    // tuning (or the defaults: square tiles, the occupancy limit)
    b->choice.xform_shape = 0;
    b->choice.ctas_per_sm = occ;
    if (!o.no_tune) {
        s = tune(b);
        if (s != ST_OK) return bail(s);
    }
    b->grid = b->choice.ctas_per_sm * b->sm_count;
    *out = b;
    return ST_OK;
}

extern "C" st_status st_batch_solve(st_batch* b, const void* const* F, const void* const* psi0, void* const* psi,
                                    st_solve_info* infos, void* stream) {
    if (!b) return fail(ST_ERR_ARG, "st_batch_solve: NULL plan");
    if (!F || !psi) return fail(ST_ERR_ARG, "st_batch_solve: NULL array");
    const int P = b->P;
    for (int p = 0; p < P; ++p) {
        if (!F[p] || !psi[p]) return fail(ST_ERR_ARG, "st_batch_solve: NULL F or psi");
        if (F[p] == psi[p]) return fail(ST_ERR_ARG, "st_batch_solve: psi must not alias F");
    }
    DevGuard guard(b->device);
    cudaStream_t us = reinterpret_cast<cudaStream_t>(stream);
    cudaStream_t st = b->cs;
    BT_TRY(cudaEventRecord(b->ev_in, us));
    BT_TRY(cudaStreamWaitEvent(st, b->ev_in, 0));
    // per-call pointers into the descriptors; psi is the iterate (psi_hat), psi0 added at the end
    long long sp = 0;
    for (int p = 0; p < P; ++p) {
        BatchProb& pr = b->hprob[p];
        const st_fdm* h = b->hs[p];
        pr.F = static_cast<const double2*>(F[p]);
        pr.x = static_cast<double2*>(psi[p]);
        pr.apsi0 = nullptr;
        if (psi0 && psi0[p]) {
            double2* a = b->apsi0 + sp;
            BT_TRY(launch_stencil_A(h->sm, psi0[p], false, nullptr, 1.0, a, st));
            pr.apsi0 = a;
        }
        sp += h->sm.n_x;
        BT_TRY(cudaMemsetAsync(psi[p], 0, (size_t)pr.n_t * pr.n_x * sizeof(double2), st));
    }
    BT_TRY(cudaMemcpyAsync(b->d_prob, b->hprob.data(), sizeof(BatchProb) * P, cudaMemcpyHostToDevice, st));
    BT_TRY(cudaMemsetAsync(b->status, 0, 2 * sizeof(int), st));
    BT_TRY(cudaMemsetAsync(b->factored, 0, sizeof(int) * P, st));   // this call's right-hand sides: factor anew
    BT_TRY(kb_launch_init(b->gm, P, b->m, st));
    if (b->use_graph) {
        st_status s = build_graph(b);
        if (s != ST_OK) return s;
    }
    // restart cycles until no problem is left iterating
    b->cycles = 0;
    const int max_cycles = b->maxit + 2;
    for (;;) {
        if (b->use_graph) BT_TRY(cudaGraphLaunch(b->exec, st));
        else BT_TRY(enqueue_cycle(b, st));
        ++b->cycles;
        int pending = 0;
        BT_TRY(cudaMemcpyAsync(&pending, b->gm.pending, sizeof(int), cudaMemcpyDeviceToHost, st));
        BT_TRY(cudaStreamSynchronize(st));
        if (pending == 0 || b->cycles >= max_cycles) break;
    }
    for (int p = 0; p < P; ++p)
        if (psi0 && psi0[p])
            BT_TRY(launch_add_row(b->hprob[p].n_t, b->hprob[p].n_x, psi[p], psi0[p], false, st));
    // per-problem outcome
    std::vector<int> stopped(P), its(P), nh(P);
    std::vector<double> rel(P), hist((size_t)P * 16);
    int flag[2] = {0, 0};
    BT_TRY(cudaMemcpyAsync(stopped.data(), b->gm.stopped, P * sizeof(int), cudaMemcpyDeviceToHost, st));
    BT_TRY(cudaMemcpyAsync(its.data(), b->gm.its, P * sizeof(int), cudaMemcpyDeviceToHost, st));
    BT_TRY(cudaMemcpyAsync(nh.data(), b->gm.nh, P * sizeof(int), cudaMemcpyDeviceToHost, st));
    BT_TRY(cudaMemcpyAsync(rel.data(), b->gm.rel, P * sizeof(double), cudaMemcpyDeviceToHost, st));
    BT_TRY(cudaMemcpyAsync(hist.data(), b->gm.hist, (size_t)P * 16 * sizeof(double), cudaMemcpyDeviceToHost, st));
    BT_TRY(cudaMemcpyAsync(flag, b->status, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    BT_TRY(cudaStreamSynchronize(st));
    BT_TRY(cudaEventRecord(b->ev_out, st));
    BT_TRY(cudaStreamWaitEvent(us, b->ev_out, 0));
    int bad = -1;
    for (int p = 0; p < P; ++p) {
        if (infos) {
            st_solve_info& inf = infos[p];
            const st_fdm* h = b->hs[p];
            inf.sweeps = its[p];
            inf.factors_kept = 0;
            inf.restart = b->m;
            inf.kept_systems = 0;
            inf.reorth_steps = 0;
            inf.rel_error_estimate = -1;
            inf.rel_residual = rel[p];
            for (int i = 0; i < 16; ++i) inf.residual_history[i] = (i < nh[p]) ? hist[(size_t)p * 16 + i] : -1.0;
            inf.kappa_x = h->td.kappa;
            inf.min_neg_im_shift = h->td.min_neg_im;
            inf.setup_seconds = h->setup_seconds;
            inf.tensor_cores = 0;
            inf.kernel_launches = 0;
        }
        if (stopped[p] != 1 && bad < 0) bad = p;
    }
    if (flag[0]) return fail(ST_ERR_ZERO_PIVOT, "st_batch_solve: zero or non-finite pivot in a spatial solve");
    if (bad >= 0)
        return fail(ST_ERR_NOT_CONVERGED, "st_batch_solve: problem " + std::to_string(bad) +
                                              (stopped[bad] == 3 ? " has a non-finite residual"
                                                                 : " did not reach the tolerance in max_sweeps"));
    return ST_OK;
}

extern "C" st_status st_batch_spatial_solve(st_batch* b, void* stream) {
    if (!b) return fail(ST_ERR_ARG, "st_batch_spatial_solve: NULL plan");
    DevGuard guard(b->device);
    cudaStream_t us = reinterpret_cast<cudaStream_t>(stream);
    BT_TRY(cudaMemsetAsync(b->status, 0, 2 * sizeof(int), us));
    BT_TRY(band_batch_launch(b->d_band, b->d_items, b->n_items, nullptr, nullptr, b->counter, b->b_max, b->win, b->Lslots,
                             b->L_stride, b->Dslots, b->D_stride, b->status, b->grid, us));
    return ST_OK;
}

extern "C" st_status st_batch_spatial_get(const st_batch* b, int p, void* G, int to_plan, void* stream) {
    if (!b || !G || p < 0 || p >= b->P) return fail(ST_ERR_ARG, "st_batch_spatial_get: bad argument");
    DevGuard guard(b->device);
    const size_t bytes = (size_t)b->hprob[p].n_t * b->hprob[p].n_x * sizeof(float2);
    float2* slot = b->G + b->off[p];
    BT_TRY(cudaMemcpyAsync(to_plan ? static_cast<void*>(slot) : G, to_plan ? G : static_cast<const void*>(slot), bytes,
                           cudaMemcpyDeviceToDevice, reinterpret_cast<cudaStream_t>(stream)));
    return ST_OK;
}

extern "C" st_status st_batch_stats_get(const st_batch* b, st_batch_stats* out) {
    if (!b || !out) return fail(ST_ERR_ARG, "st_batch_stats_get: NULL argument");
    std::memset(out, 0, sizeof(*out));
    out->count = b->P;
    out->items = b->n_items;
    out->restart = b->m;
    int bm = 0, bn = 0;
    kb_xform_shape(b->choice.xform_shape, &bm, &bn);
    out->xform_tile_m = bm;
    out->xform_tile_n = bn;
    out->solve_ctas_per_sm = b->choice.ctas_per_sm;
    out->solve_grid = b->grid;
    out->graph_nodes = (int)b->graph_nodes;
    out->cycles = b->cycles;
    out->tuned = b->tuned;
    out->tune_seconds = b->tune_seconds;
    out->unknowns = b->N;
    out->workspace_bytes = (unsigned long long)b->bytes;
    out->kept_problems = b->kept;
    out->kept_factor_bytes = (unsigned long long)b->kept_bytes;
    return ST_OK;
}

extern "C" void st_destroy_batch(st_batch* b) { destroy(b); }

// One-shot batched solve.  ST_MIXED: a plan as above (the tuner's choice is cached per shape
// signature, so repeated calls with the same shapes do not retune).  ST_FP64 / ST_FP32, and the
// classic or fixed-sweep refinement variants: the problems are solved one after another.
extern "C" st_status st_fdm_solve_batched(st_fdm* const* hs, int count, const void* const* F,
                                          const void* const* psi0, void* const* psi, const st_solve_opts* opts,
                                          st_solve_info* infos, void* stream) {
    if (count < 0 || (count > 0 && (!hs || !F || !psi))) return fail(ST_ERR_ARG, "st_fdm_solve_batched: bad arguments");
    if (count == 0) return ST_OK;
    const bool grouped = opts && opts->precision == ST_MIXED && opts->fixed_sweeps <= 0 &&
                         opts->method == ST_REFINE_GMRES;
    if (!grouped) {
        for (int i = 0; i < count; ++i) {
            st_status s = st_fdm_solve(hs[i], F[i], psi0 ? psi0[i] : nullptr, psi[i], opts,
                                       infos ? &infos[i] : nullptr, stream);
            if (s != ST_OK) return s;
        }
        return ST_OK;
    }
    st_batch_opts bo;
    std::memset(&bo, 0, sizeof(bo));
    bo.tol = opts->tol;
    bo.max_sweeps = opts->max_sweeps;
    st_batch* b = nullptr;
    st_status s = st_batch_create(hs, count, &bo, &b);
    if (s != ST_OK) return s;
    s = st_batch_solve(b, F, psi0, psi, infos, stream);
    st_destroy_batch(b);
    return s;
}
