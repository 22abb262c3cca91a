// Batched Chebyshev filtering (CheFSI, Sec. II.B) of many independent systems -- AIMD
// snapshots, Bloch wavevectors, spin channels of uneven grid and orbital counts -- in one
// CUDA graph, plus the autotuner that picks each system's stencil tile shape and the
// split factor of the tensor-core Gram products.
//
// The graph holds one chain per system (fork / join through events), so the GPU runs the
// chains concurrently and small systems fill the machine together.  Every kernel of a
// chain reads its recurrence coefficients {alpha, beta, shift} for its degree from a device
// table, so a cached graph is replayed for new filter bounds after one host-to-device copy.
#include <algorithm>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>

#include "hub_internal.cuh"

namespace hub {

namespace {

struct TuneKey {
    int n1, n2, n3, ncol, esize, cplx;
    bool operator<(const TuneKey& o) const {
        return std::tie(n1, n2, n3, ncol, esize, cplx) < std::tie(o.n1, o.n2, o.n3, o.ncol, o.esize, o.cplx);
    }
};
std::mutex g_tune_mu;
struct TuneVal {
    int variant, split, gather_form;
};
std::map<TuneKey, TuneVal> g_tuned;   // shape -> stencil variant, gemm split, gather form

struct BatchGraph {
    std::vector<hub_t> sys;
    std::vector<int> spin, ncol, ld;
    std::vector<void*> X;
    int degree = 0;
    cudaStream_t origin = nullptr;
    cudaGraphExec_t exec = nullptr;
    double* d_coef = nullptr;
    double* h_coef = nullptr;          // pinned staging for the coefficient table
    cudaStream_t launch = nullptr;     // captured and replayed here (the caller's stream may be
                                       // the legacy default stream, which cannot be captured)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    std::vector<long long> launches;   // kernels per system and replay
    std::vector<long long> gen;        // memory generation of every handle at capture
    int lanes = 1;
    ~BatchGraph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (d_coef) cudaFree(d_coef);
        if (h_coef) cudaFreeHost(h_coef);
        for (auto s : streams) cudaStreamDestroy(s);
        for (auto e : events) cudaEventDestroy(e);
        if (launch) cudaStreamDestroy(launch);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
    }
    bool matches(int n, const hub_t* s, const int* sp, void* const* x, const int* nc, const int* l, int deg,
                 cudaStream_t st) const {
        if ((int)sys.size() != n || degree != deg || origin != st) return false;
        for (int i = 0; i < n; ++i)
            if (sys[i] != s[i] || spin[i] != sp[i] || X[i] != x[i] || ncol[i] != nc[i] || ld[i] != l[i] ||
                gen[i] != s[i]->mem_gen)
                return false;
        return true;
    }
};
std::mutex g_batch_mu;
std::vector<std::unique_ptr<BatchGraph>> g_batches;   // a few recent graphs

// X <- p_m(H) X with coefficients read on the device: coef[3k .. 3k+2] for degree k + 1
int filter_chain(hub_t h, int spin, void* X, int ncol, int ld, int degree, const double* coef) {
    int rc;
    void* B1 = h->d_work;
    if ((rc = apply_H_internal(h, spin, X, ld, B1, ncol, 1.0, 0.0, nullptr, 0.0, coef))) return rc;
    void* cur = B1;
    void* prev = X;
    for (int k = 1; k < degree; ++k) {
        if ((rc = apply_H_internal(h, spin, cur, ld, prev, ncol, 1.0, 0.0, prev, 0.0, coef + 3 * k))) return rc;
        std::swap(cur, prev);
    }
    if (cur != X)
        if ((rc = launch_copy_block(h, cur, ld, X, ld, ncol))) return rc;
    return HUB_OK;
}

void filter_coefficients(int degree, double a, double b, double a_low, double* out) {
    const double e = 0.5 * (b - a), c = 0.5 * (b + a);
    double sigma = e / (a_low - c);
    const double tau = 2.0 / sigma;
    out[0] = sigma / e;
    out[1] = 0.0;
    out[2] = c;
    for (int k = 1; k < degree; ++k) {
        const double sn = 1.0 / (tau - sigma);
        out[3 * k] = 2.0 * sn / e;
        out[3 * k + 1] = -sigma * sn;
        out[3 * k + 2] = c;
        sigma = sn;
    }
}

}  // namespace

}  // namespace hub

using namespace hub;

#define BATCH_TRY(expr)                                                                    \
    do {                                                                                   \
        cudaError_t _e = (expr);                                                           \
        if (_e != cudaSuccess)                                                             \
            return hub::fail(sys[0], HUB_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
    } while (0)

extern "C" {

int hub_set_tuning(hub_t h, int stencil_variant, int gemm_split, int gather_form) {
    if (!h) return HUB_EINVAL;
    if (stencil_variant >= hub::stencil_variants(h) || stencil_variant < -1 || gemm_split == 0 || gemm_split < -1 ||
        gather_form < -1 || gather_form > 3 || (gather_form >= 1 && (h->esize != 4 || h->cplx)) ||
        (gather_form >= 2 && !h->proj.tc))
        return hub::fail(h, HUB_EINVAL, "bad tuning");
    if (stencil_variant >= 0) h->stencil_variant = stencil_variant;
    if (gemm_split > 0) h->gemm_split = gemm_split;
    if (gather_form >= 0) h->gather_dense = gather_form;
    return HUB_OK;
}

int hub_get_tuning(hub_t h, int* stencil_variant, int* n_variants, int* gemm_split, int* gather_form) {
    if (!h) return HUB_EINVAL;
    if (stencil_variant) *stencil_variant = h->stencil_variant;
    if (n_variants) *n_variants = hub::stencil_variants(h);
    if (gemm_split) *gemm_split = h->gemm_split;
    if (gather_form) *gather_form = h->gather_dense;
    return HUB_OK;
}

int hub_autotune(hub_t h, int spin, const void* X, int ncol, int ld, int* variant_out) {
    if (!h || !X || ncol < 1 || (long)ld < h->Nd) return hub::fail(h, HUB_EINVAL, "bad autotune arguments");
    if (!h->veff_set || !h->atoms_set) return hub::fail(h, HUB_EINVAL, "handle not set up");
    const TuneKey key{h->n1, h->n2, h->n3, ncol, h->esize, h->cplx};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            h->stencil_variant = it->second.variant;
            h->gemm_split = it->second.split;
            h->gather_dense = (h->proj.dense && h->esize == 4 && !h->cplx &&
                               (it->second.gather_form < 2 || h->proj.tc)) ? it->second.gather_form : 0;
            if (variant_out) *variant_out = h->stencil_variant;
            return HUB_OK;
        }
    }
    int rc;
    const size_t es = (size_t)h->esize * (h->cplx ? 2 : 1);
    if ((rc = ensure(h, &h->d_work, &h->work_bytes, std::max(h->work_bytes, (size_t)ld * ncol * es)))) return rc;
    // one application first: sizes the gather workspaces, warms the caches
    if ((rc = apply_H_internal(h, spin, X, ld, h->d_work, ncol, 1.0, 0.0, nullptr, 0.0))) return rc;
    cudaEvent_t e0, e1;
    HUB_CUDA_TRY(h, cudaEventCreate(&e0));
    HUB_CUDA_TRY(h, cudaEventCreate(&e1));
    // stencil tile shape: time the stencil kernel alone, best of 3 launches per candidate
    StencilArgs a{};
    {
        double c0 = 0.0;
        a.Y = X; a.Yprev = nullptr; a.Yout = h->d_work; a.V = h->d_veff;
        a.n1 = h->n1; a.n2 = h->n2; a.n3 = h->n3; a.ld = ld; a.ncol = ncol; a.n0 = h->n0;
        // Laplacian weights of order 2 n0 (same closed form as apply_H)
        auto fact = [](int k) { double r = 1.0; for (int i = 2; i <= k; ++i) r *= i; return r; };
        double csum = 0.0, inv2 = 0.0;
        for (int p = 1; p <= h->n0; ++p) csum += 1.0 / ((double)p * p);
        c0 = -2.0 * csum;
        for (int ax = 0; ax < 3; ++ax) {
            const double ih2 = 1.0 / (h->h[ax] * h->h[ax]);
            inv2 += ih2;
            for (int p = 1; p <= h->n0; ++p) {
                const double cp = 2.0 * ((p % 2) ? 1.0 : -1.0) * fact(h->n0) * fact(h->n0) /
                                  ((double)p * p * fact(h->n0 - p) * fact(h->n0 + p));
                a.w[ax][p - 1] = -0.5 * cp * ih2;
                a.wbase[ax][p - 1] = a.w[ax][p - 1];
            }
            a.phase[ax][0] = std::cos(h->kpt[ax] * h->L[ax]);
            a.phase[ax][1] = std::sin(h->kpt[ax] * h->L[ax]);
        }
        a.center = -0.5 * c0 * inv2;
        a.alpha = 1.0;
        a.beta = 0.0;
        a.coef = nullptr;
    }
    const int nv = stencil_variants(h);
    int best = 0;
    float best_ms = 1e30f;
    const int saved_prof = h->prof_on;
    h->prof_on = 0;
    for (int v = 0; v < nv; ++v) {
        h->stencil_variant = v;
        if ((rc = launch_stencil(h, a))) { h->prof_on = saved_prof; return rc; }   // warm-up
        float ms_min = 1e30f;
        for (int r = 0; r < 3; ++r) {
            HUB_CUDA_TRY(h, cudaEventRecord(e0, h->stream));
            if ((rc = launch_stencil(h, a))) { h->prof_on = saved_prof; return rc; }
            HUB_CUDA_TRY(h, cudaEventRecord(e1, h->stream));
            HUB_CUDA_TRY(h, cudaEventSynchronize(e1));
            float ms = 0.f;
            HUB_CUDA_TRY(h, cudaEventElapsedTime(&ms, e0, e1));
            ms_min = std::min(ms_min, ms);
        }
        if (ms_min < best_ms) { best_ms = ms_min; best = v; }
    }
    h->stencil_variant = best;
    // split factor of the tensor-core Gram product (mixed handles, real float blocks)
    int best_split = h->gemm_split;
    if ((h->prec == HUB_MIXED_BF16 || h->prec == HUB_MIXED_F16) && !h->cplx && ncol >= 16) {
        const size_t gb = (size_t)ncol * ncol * sizeof(double);
        if ((rc = ensure(h, &h->d_small, &h->small_bytes, std::max(h->small_bytes, gb)))) { h->prof_on = saved_prof; return rc; }
        float bms = 1e30f;
        const int saved_terms = h->bf16_terms;
        h->bf16_terms = 3;
        for (int sp : {1, 2, 4}) {
            h->gemm_split = sp;
            if ((rc = launch_gram_bf16(h, X, ld, h->d_work, ld, ncol, ncol, 1.0, false, (double*)h->d_small))) break;
            HUB_CUDA_TRY(h, cudaEventRecord(e0, h->stream));
            rc = launch_gram_bf16(h, X, ld, h->d_work, ld, ncol, ncol, 1.0, false, (double*)h->d_small);
            HUB_CUDA_TRY(h, cudaEventRecord(e1, h->stream));
            HUB_CUDA_TRY(h, cudaEventSynchronize(e1));
            if (rc) break;
            float ms = 0.f;
            HUB_CUDA_TRY(h, cudaEventElapsedTime(&ms, e0, e1));
            if (ms < bms) { bms = ms; best_split = sp; }
        }
        h->bf16_terms = saved_terms;
        if (rc) { h->prof_on = saved_prof; return rc; }
    }
    h->gemm_split = best_split;
    // projector forms (real float handles with brick tables), gather and scatter timed
    // together: point-major; bricks on CUDA cores; the tensor-core gather with the CUDA-core
    // scatter; both on the tensor cores
    int best_form = 0;
    if (h->proj.dense && h->esize == 4 && !h->cplx) {
        float fms[4] = {1e30f, 1e30f, 1e30f, 1e30f};
        const int nforms = h->proj.tc ? 4 : 2;
        for (int form = 0; form < nforms && !rc; ++form) {
            h->gather_dense = form;
            if ((rc = launch_gather(h, X, ncol, ld, spin, true))) break;       // warm-up
            if ((rc = launch_scatter(h, h->d_work, ncol, ld, 1.0))) break;
            for (int r = 0; r < 3 && !rc; ++r) {
                HUB_CUDA_TRY(h, cudaEventRecord(e0, h->stream));
                rc = launch_gather(h, X, ncol, ld, spin, true);
                if (!rc) rc = launch_scatter(h, h->d_work, ncol, ld, 1.0);
                HUB_CUDA_TRY(h, cudaEventRecord(e1, h->stream));
                HUB_CUDA_TRY(h, cudaEventSynchronize(e1));
                float ms = 0.f;
                HUB_CUDA_TRY(h, cudaEventElapsedTime(&ms, e0, e1));
                fms[form] = std::min(fms[form], ms);
            }
        }
        if (rc) { h->prof_on = saved_prof; return rc; }
        for (int form = 1; form < nforms; ++form)
            if (fms[form] < fms[best_form]) best_form = form;
    }
    h->gather_dense = best_form;
    h->prof_on = saved_prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key] = {best, best_split, best_form};
    }
    if (variant_out) *variant_out = best;
    return check_flags(h);
}

int hub_batch_filter(int nsys, const hub_t* sys, const int* spin, void* const* X, const int* ncol,
                     const int* ld, int degree, const double* a, const double* b, const double* a_low,
                     void* cuda_stream) {
    hub::NvtxRange nvtx_("hub_batch_filter");
    if (nsys < 1 || !sys || !spin || !X || !ncol || !ld || !a || !b || !a_low || degree < 1) return HUB_EINVAL;
    int dev = -1;
    BATCH_TRY(cudaGetDevice(&dev));
    for (int i = 0; i < nsys; ++i) {
        hub_t h = sys[i];
        if (!h || h->device != dev) return HUB_EINVAL;
        if (!h->veff_set || !h->atoms_set) return hub::fail(h, HUB_EINVAL, "handle not set up");
        if (spin[i] < 0 || spin[i] > 1 || ncol[i] < 1 || (long)ld[i] < h->Nd || !X[i])
            return hub::fail(h, HUB_EINVAL, "bad block of a batched system");
        if (!(a_low[i] < a[i] && a[i] < b[i])) return hub::fail(h, HUB_EINVAL, "filter bounds need a_low < a < b");
        for (int j = 0; j < i; ++j)
            if (sys[j] == h) return hub::fail(h, HUB_EINVAL, "a handle appears twice in one batch");
    }
    cudaStream_t origin = (cudaStream_t)cuda_stream;
    std::lock_guard<std::mutex> lk(g_batch_mu);
    BatchGraph* G = nullptr;
    for (size_t k = 0; k < g_batches.size(); ++k) {
        auto& g = g_batches[k];
        if (g->matches(nsys, sys, spin, X, ncol, ld, degree, origin)) { G = g.get(); break; }
        // a graph over the same handles whose workspaces moved can never be replayed again
        bool stale = false;
        for (size_t i = 0; i < g->sys.size(); ++i)
            for (int j = 0; j < nsys; ++j)
                if (g->sys[i] == sys[j] && g->gen[i] != sys[j]->mem_gen) stale = true;
        if (stale) { g_batches.erase(g_batches.begin() + k); --k; }
    }
    if (!G) {
        auto g = std::make_unique<BatchGraph>();
        g->sys.assign(sys, sys + nsys);
        g->spin.assign(spin, spin + nsys);
        g->X.assign(X, X + nsys);
        g->ncol.assign(ncol, ncol + nsys);
        g->ld.assign(ld, ld + nsys);
        g->degree = degree;
        g->origin = origin;
        const size_t cbytes = (size_t)nsys * degree * 3 * sizeof(double);
        BATCH_TRY(cudaMalloc(&g->d_coef, cbytes));
        BATCH_TRY(cudaMallocHost(&g->h_coef, cbytes));
        // workspaces and tile shapes before capture (nothing may allocate inside it)
        for (int i = 0; i < nsys; ++i) {
            hub_t h = sys[i];
            const size_t es = (size_t)h->esize * (h->cplx ? 2 : 1);
            int rc;
            // one real application sizes every workspace the chain touches (the tuning cache
            // may skip the autotuner's own application for shapes seen before)
            if ((rc = ensure(h, &h->d_work, &h->work_bytes, std::max(h->work_bytes, (size_t)ld[i] * ncol[i] * es))) ||
                (rc = apply_H_internal(h, spin[i], X[i], ld[i], h->d_work, ncol[i], 1.0, 0.0, nullptr, 0.0)) ||
                (rc = hub_autotune(h, spin[i], X[i], ncol[i], ld[i], nullptr))) {
                if (h != sys[0]) sys[0]->last_error = "system " + std::to_string(i) + ": " + h->last_error;
                return rc;
            }
        }
        BATCH_TRY(cudaStreamCreateWithFlags(&g->launch, cudaStreamNonBlocking));
        BATCH_TRY(cudaEventCreateWithFlags(&g->ev_in, cudaEventDisableTiming));
        BATCH_TRY(cudaEventCreateWithFlags(&g->ev_out, cudaEventDisableTiming));
        // lanes: chains inside a lane run one after another, lanes run concurrently.  A
        // system whose H application fills the GPU by itself gains nothing from running
        // beside others (they only evict each other's L2 lines), small ones fill it together.
        double total = 0.0;
        for (int i = 0; i < nsys; ++i) total += (double)sys[i]->Nd * ncol[i];
        const double fill = 2048.0 * 32.0 * sys[0]->num_sms;          // point-orbitals
        int lanes = (int)std::lround(2.0 * fill * nsys / std::max(total, 1.0));
        lanes = std::max(1, std::min(nsys, lanes));
        std::vector<int> order(nsys);
        for (int i = 0; i < nsys; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            return (double)sys[x]->Nd * ncol[x] > (double)sys[y]->Nd * ncol[y];
        });
        g->streams.resize(lanes);
        g->events.resize(lanes + 1);
        for (int l = 0; l < lanes; ++l) BATCH_TRY(cudaStreamCreateWithFlags(&g->streams[l], cudaStreamNonBlocking));
        for (auto& e : g->events) BATCH_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        BATCH_TRY(cudaDeviceSynchronize());
        g->gen.resize(nsys);
        for (int i = 0; i < nsys; ++i) g->gen[i] = sys[i]->mem_gen;
        cudaGraph_t graph;
        BATCH_TRY(cudaStreamBeginCapture(g->launch, cudaStreamCaptureModeThreadLocal));
        int crc = HUB_OK;
        cudaEventRecord(g->events[lanes], g->launch);
        for (int l = 0; l < lanes; ++l) cudaStreamWaitEvent(g->streams[l], g->events[lanes], 0);
        g->launches.assign(nsys, 0);
        for (int k = 0; k < nsys && !crc; ++k) {
            const int i = order[k];
            hub_t h = sys[i];
            cudaStream_t saved = h->stream;
            h->stream = g->streams[k % lanes];
            h->capturing = 1;
            const long long l0 = h->launches;
            crc = filter_chain(h, spin[i], X[i], ncol[i], ld[i], degree, g->d_coef + (size_t)i * degree * 3);
            g->launches[i] = h->launches - l0;
            h->launches = l0;
            h->capturing = 0;
            h->stream = saved;
        }
        for (int l = 0; l < lanes; ++l) {
            cudaEventRecord(g->events[l], g->streams[l]);
            cudaStreamWaitEvent(g->launch, g->events[l], 0);
        }
        g->lanes = lanes;
        const cudaError_t ec = cudaStreamEndCapture(g->launch, &graph);
        if (crc) {
            for (int i = 1; i < nsys; ++i)
                if (!sys[i]->last_error.empty()) sys[0]->last_error = "capture, system " + std::to_string(i) + ": " + sys[i]->last_error;
            return crc;
        }
        if (ec != cudaSuccess) return hub::fail(sys[0], HUB_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
        const cudaError_t ei = cudaGraphInstantiate(&g->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) return hub::fail(sys[0], HUB_ECUDA, std::string("graph instantiation: ") + cudaGetErrorString(ei));
        if (g_batches.size() >= 4) g_batches.erase(g_batches.begin());
        g_batches.push_back(std::move(g));
        G = g_batches.back().get();
    }
    for (int i = 0; i < nsys; ++i) filter_coefficients(degree, a[i], b[i], a_low[i], G->h_coef + (size_t)i * degree * 3);
    // order: caller's stream -> coefficient copy + graph on the launch stream -> caller's stream
    BATCH_TRY(cudaEventRecord(G->ev_in, origin));
    BATCH_TRY(cudaStreamWaitEvent(G->launch, G->ev_in, 0));
    BATCH_TRY(cudaMemcpyAsync(G->d_coef, G->h_coef, (size_t)nsys * degree * 3 * sizeof(double),
                              cudaMemcpyHostToDevice, G->launch));
    BATCH_TRY(cudaGraphLaunch(G->exec, G->launch));
    BATCH_TRY(cudaEventRecord(G->ev_out, G->launch));
    BATCH_TRY(cudaStreamWaitEvent(origin, G->ev_out, 0));
    for (int i = 0; i < nsys; ++i) sys[i]->launches += G->launches[i];
    // the pinned coefficient table is reused by the next call: it must not change before
    // this copy has run
    BATCH_TRY(cudaStreamSynchronize(G->launch));
    return HUB_OK;
}

}  // extern "C"
