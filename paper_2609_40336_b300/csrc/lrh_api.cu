// Host side of the C ABI declared in include/lrh.h: region poset (covering pairs of the
// inclusion order, Sec. 4.2), term placement and embedding, device state, and the
// iteration driver (per-iteration kernel sequence, optionally replayed as a CUDA graph).
#include "../../include/lrh.h"
#include "lrh_internal.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <limits>
#include <memory>
#include <new>
#include <set>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

using namespace lrh;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

#define LRH_CK(call)                                                                           \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(LRH_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));        \
    } while (0)

struct VecHash {
    size_t operator()(const std::vector<int32_t>& v) const {
        uint64_t h = 1469598103934665603ull;
        for (int32_t x : v) { h ^= (uint64_t)(uint32_t)x; h *= 1099511628211ull; }
        return (size_t)h;
    }
};

constexpr int kMaxSites = 8;     // region size limit of the data layout (D <= 256)
constexpr int kMaxKernelSites = 8;  // sizes with a region-pass kernel in this build (D <= 256)
constexpr int kBigLogSweeps = 16;   // FP32 sweep cap of 8-site regions (their rotation log holds 16 sweeps)
constexpr int kGraphChunk = 8;   // iterations per captured graph (even: parity returns to 0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev); else prev = -1;
    }
    ~DeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

}  // namespace

int lrh::set_last_error(int code, const std::string& msg) { return fail(code, msg); }

struct lrh_problem {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    lrh_options opt{};
    std::vector<double> beta_sched;   // owned copies of the options' host arrays
    std::string tune_cache;
    std::vector<double> target;
    int32_t n_sites = 0, kappa = 0;
    double lhat_eff = 1.0;
    int32_t n_inst = 1, n_regions = 0, n_pairs = 0, max_k = 0;
    int64_t msg_elems = 0, h_elems = 0, rho_elems = 0;
    double lambda_G = 0, gamma_G = 0;
    int64_t iteration = 0;
    bool stepped_since_restart = false;
    std::vector<int32_t> pair_parent, pair_child;
    std::vector<int64_t> pair_off;
    // size classes: k -> device list of region ids
    std::vector<int> class_k;
    std::vector<int32_t> class_count;
    std::vector<int32_t*> class_list;
    // device memory
    DevProblem P{};
    std::vector<void*> allocs;
    double* h_pinned = nullptr;   // host staging for bound / values
    int64_t h_pinned_len = 0;
    cudaGraph_t graph = nullptr;            // Alg. 1: graph of kGraphChunk iterations
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<std::pair<int, cudaGraphExec_t>> nest_graphs;   // Alg. 2: one per n_iters
    // term structure (for lrh_set_terms and the adjoint)
    int32_t n_terms = 0;
    int64_t term_total = 0;
    std::vector<int32_t> term_region, term_mask, term_kt;
    std::vector<int64_t> term_off, region_h_off;
    std::vector<int32_t> region_k;
    int64_t all_elems = 0;
    float2* vjp_nubar = nullptr;    // adjoint outputs staged on the device
    float2* vjp_termbar = nullptr;
    float2* vjp_scratch = nullptr;  // CTA adjoint (6-7 sites): one slot of 2 D^2 complex per CTA
    int vjp_slots = 0;
    // region classes after the first run on forked streams (joined before the update)
    std::vector<cudaStream_t> aux;
    std::vector<cudaEvent_t> ev_join;
    cudaEvent_t ev_fork = nullptr;
    // launch shape per class (threads per CTA of the lane kernels) and stream concurrency,
    // chosen by lrh_autotune (defaults: 128 threads, concurrent classes)
    std::vector<int> class_block;
    bool concurrent = true;
    bool fused = false;   // all classes (<= 4 sites) in one launch per pass (autotuned)
    // persistent driver: plan of the cooperative launch (classes with k <= 4 only), its grid,
    // the resident-CTA capacity and the autotuned driver for LRH_LOOP_AUTO (-1: not tuned)
    PersistPlan plan{};
    int persist_kmax = 0;
    int persist_grid = 0;
    int64_t persist_cap = 0;
    int loop_auto = -1;
    // sharding with halo exchange: ghost regions (pass run by another shard) and the exchange maps
    // of lrh_halo_set (per 4-entry chunk of one instance's buffer: offset in the state arena, or
    // ~offset in the partial-trace arena)
    std::vector<uint8_t> ghost;
    bool has_ghost = false;
    int64_t* halo_send = nullptr;
    int64_t* halo_recv = nullptr;
    int64_t halo_send_chunks = 0, halo_recv_chunks = 0;
    bool halo_ready = false;
    bool halo_passed = false;   // lrh_halo_pass ran and lrh_halo_update has not yet
    int64_t warm_elems = 0;     // complex entries of the stored eigenbases (P.warm)

    template <typename T>
    int dalloc(T** ptr, int64_t count) {
        *ptr = nullptr;
        if (count <= 0) count = 1;
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, (size_t)count * sizeof(T));
        if (e != cudaSuccess) return fail(LRH_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        allocs.push_back(p);
        *ptr = static_cast<T*>(p);
        return LRH_OK;
    }
    void dfree(void* ptr) {
        if (!ptr) return;
        allocs.erase(std::remove(allocs.begin(), allocs.end(), ptr), allocs.end());
        cudaFree(ptr);
    }
    ~lrh_problem() {
        for (auto& g : nest_graphs) cudaGraphExecDestroy(g.second);
        for (cudaStream_t a : aux) cudaStreamDestroy(a);
        for (cudaEvent_t e : ev_join) cudaEventDestroy(e);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (graph_exec) cudaGraphExecDestroy(graph_exec);
        if (graph) cudaGraphDestroy(graph);
        for (void* p : allocs) cudaFree(p);
        if (h_pinned) cudaFreeHost(h_pinned);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

namespace {

int validate_options(const lrh_options* o) {
    if (!o) return fail(LRH_EINVAL, "options is NULL");
    if (o->n_beta < 0 || (o->n_beta > 0 && !o->beta_sched)) return fail(LRH_EINVAL, "beta_sched is NULL or n_beta < 0");
    for (int i = 0; i < o->n_beta; ++i)
        if (!(o->beta_sched[i] > 0.0) || !std::isfinite(o->beta_sched[i])) return fail(LRH_EINVAL, "beta_sched entries must be finite and > 0");
    if (o->iters_per_stage < 0 || o->certify_every < 0) return fail(LRH_EINVAL, "iters_per_stage and certify_every must be >= 0");
    if (!std::isfinite(o->deadline_s)) return fail(LRH_EINVAL, "non-finite deadline_s");
    if (!(o->screen_tol >= 0.0) || !std::isfinite(o->screen_tol)) return fail(LRH_EINVAL, "screen_tol must be finite and >= 0");
    if (o->variant != LRH_SUBGRADIENT && o->variant != LRH_NESTEROV) return fail(LRH_EINVAL, "unknown variant");
    if (o->step_rule != LRH_STEP_CONST && o->step_rule != LRH_STEP_INV_SQRT) return fail(LRH_EINVAL, "unknown step rule");
    if (o->variant == LRH_SUBGRADIENT && !(o->alpha > 0.0)) return fail(LRH_EINVAL, "alpha must be > 0");
    if (o->variant == LRH_NESTEROV && !(o->beta > 0.0)) return fail(LRH_EINVAL, "beta must be > 0");
    if (!std::isfinite(o->beta) || !std::isfinite(o->alpha) || !std::isfinite(o->lhat)) return fail(LRH_EINVAL, "non-finite option");
    if (o->loop < LRH_LOOP_EAGER || o->loop > LRH_LOOP_AUTO) return fail(LRH_EINVAL, "unknown iteration driver (loop)");
    return LRH_OK;
}

// Options with their host arrays copied into the problem (the caller's may go away);
// p->n_inst must be set (the length of `target`).
void copy_options(lrh_problem* p, const lrh_options* o) {
    p->opt = *o;
    p->beta_sched.assign(o->beta_sched, o->beta_sched + (o->n_beta > 0 ? o->n_beta : 0));
    p->opt.beta_sched = p->beta_sched.empty() ? nullptr : p->beta_sched.data();
    p->tune_cache = o->tune_cache ? o->tune_cache : "";
    p->opt.tune_cache = o->tune_cache ? p->tune_cache.c_str() : nullptr;
    if (o->target) p->target.assign(o->target, o->target + p->n_inst); else p->target.clear();
    p->opt.target = p->target.empty() ? nullptr : p->target.data();
}

int push_state(lrh_problem* p, bool set_theta_t, double theta, double t) {
    const lrh_options& o = p->opt;
    p->lhat_eff = o.lhat > 0.0 ? o.lhat : (o.beta > 0.0 ? o.beta * p->lambda_G / 2.0 : 1.0);
    const double degen = o.degen_tol > 0.0 ? o.degen_tol : 1e-5;
    const int sweeps = o.max_sweeps > 0 ? o.max_sweeps : 15;
    const int cert = o.cert_sweeps > 0 ? o.cert_sweeps : 40;
    LRH_CK(launch_set_state(p->P, (int)(p->iteration & 1), theta, t, set_theta_t ? 1 : 0, o.beta,
                            1.0 / p->lhat_eff, o.alpha, degen, o.variant, o.step_rule, sweeps, cert,
                            o.cold_start ? 1 : 0, p->stream));
    return LRH_OK;
}

// every stored eigenbasis back to the identity (the state at creation)
int reset_warm(lrh_problem* p) {
    for (size_t c = 0; c < p->class_k.size(); ++c) {
        const int k = p->class_k[c];
        if (p->P.warm && p->P.warm_off[k] >= 0)
            LRH_CK(launch_warm_identity(p->P.warm + p->P.warm_off[k], (int64_t)p->n_inst * p->class_count[c], 1 << k,
                                        p->stream));
    }
    return LRH_OK;
}

// Hermitian part of every term matrix (exactly: (m + m^dagger)/2) embedded into the dense
// region terms h_e in FP64, instance-major, at the offsets of region_h_off.
// fn(lo, hi) over [0, n) split into contiguous ranges on the host's cores (disjoint outputs)
void parallel_ranges(int64_t n, const std::function<void(int64_t, int64_t)>& fn) {
    const int64_t hw = std::max<int64_t>(1, std::min<int64_t>((int64_t)std::thread::hardware_concurrency(), 32));
    const int64_t nt = std::min<int64_t>(hw, n);
    if (nt <= 1) { fn(0, n); return; }
    std::vector<std::thread> th;
    for (int64_t w = 0; w < nt; ++w) th.emplace_back(fn, n * w / nt, n * (w + 1) / nt);
    for (auto& x : th) x.join();
}

// Every term's Hermitian part embedded into its region: for each instance, the terms in order
// (each entry of h_e sums its terms in ascending t, whatever the split over instances).
void embed_terms(const lrh_problem* p, const double* term_mats, std::vector<double>& h64) {
    auto pext = [](int x, int m) { int r = 0, q = 0; for (int bb = 0; bb < 8; ++bb) if (m >> bb & 1) { r |= (x >> bb & 1) << q; ++q; } return r; };
    h64.assign((size_t)(2 * p->n_inst * std::max<int64_t>(p->h_elems, 1)), 0.0);
    // per term, its entries (i, j) of h_e with the term entries (a, c) and (c, a) they take
    struct Ent { int32_t hij, ac, ca; bool diag; };
    std::vector<std::vector<Ent>> ents((size_t)p->n_terms);
    for (int t = 0; t < p->n_terms; ++t) {
        const int k = p->region_k[p->term_region[t]];
        const int D = 1 << k, M = p->term_mask[t], Dt = 1 << p->term_kt[t];
        for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j) {
                if (((i ^ j) & ~M) != 0) continue;
                const int a = pext(i, M), c = pext(j, M);
                ents[t].push_back(Ent{i * D + j, a * Dt + c, c * Dt + a, a == c});
            }
    }
    parallel_ranges(p->n_inst, [&](int64_t lo, int64_t hi) {
        for (int64_t inst = lo; inst < hi; ++inst)
            for (int t = 0; t < p->n_terms; ++t) {
                const double* m = term_mats + 2 * (inst * p->term_total + p->term_off[t]);
                double* h = h64.data() + 2 * (inst * p->h_elems + p->region_h_off[p->term_region[t]]);
                for (const Ent& x : ents[t]) {
                    h[2 * x.hij] += 0.5 * (m[2 * x.ac] + m[2 * x.ca]);
                    h[2 * x.hij + 1] += x.diag ? 0.0 : 0.5 * (m[2 * x.ac + 1] - m[2 * x.ca + 1]);
                }
            }
    });
}

// FP64 terms to the device, and their FP32 copy rounded there (round to nearest, as a host cast)
int upload_terms(lrh_problem* p, const std::vector<double>& h64) {
    if (!p->h_elems) return LRH_OK;
    const int64_t n = (int64_t)p->n_inst * p->h_elems;
    LRH_CK(cudaMemcpyAsync(const_cast<double2*>(p->P.h64), h64.data(), sizeof(double2) * n, cudaMemcpyHostToDevice, p->stream));
    LRH_CK(launch_round_terms(const_cast<float2*>(p->P.h32), p->P.h64, n, p->stream));
    LRH_CK(cudaStreamSynchronize(p->stream));
    return LRH_OK;
}

int check_terms(const lrh_problem* p, const int64_t* term_ptr, const double* term_mats) {
    // per instance range: the first offending term (lowest t, then lowest instance) and its kind
    std::vector<int64_t> bad((size_t)p->n_inst, -1);
    std::vector<int> kind((size_t)p->n_inst, 0);
    parallel_ranges(p->n_inst, [&](int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; ++i)
            for (int t = 0; t < p->n_terms && bad[(size_t)i] < 0; ++t) {
                const int64_t Dt = (int64_t)1 << (term_ptr[t + 1] - term_ptr[t]);
                const double* m = term_mats + 2 * (i * p->term_total + p->term_off[t]);
                double mx = 0;
                for (int64_t a = 0; a < Dt * Dt; ++a) mx = std::max(mx, std::fabs(m[2 * a]) + std::fabs(m[2 * a + 1]));
                for (int64_t a = 0; a < Dt && bad[(size_t)i] < 0; ++a)
                    for (int64_t c = 0; c < Dt; ++c) {
                        const double dr = m[2 * (a * Dt + c)] - m[2 * (c * Dt + a)];
                        const double di = m[2 * (a * Dt + c) + 1] + m[2 * (c * Dt + a) + 1];
                        if (!std::isfinite(dr) || !std::isfinite(di)) { bad[(size_t)i] = t; kind[(size_t)i] = 1; break; }
                        if (std::fabs(dr) + std::fabs(di) > 1e-10 * std::max(1.0, mx)) { bad[(size_t)i] = t; kind[(size_t)i] = 2; break; }
                    }
            }
    });
    int64_t t0 = -1;
    int k0 = 0;
    for (int64_t i = 0; i < p->n_inst; ++i)
        if (bad[(size_t)i] >= 0 && (t0 < 0 || bad[(size_t)i] < t0)) { t0 = bad[(size_t)i]; k0 = kind[(size_t)i]; }
    if (t0 >= 0) {
        if (k0 == 1) return fail(LRH_EINVAL, "non-finite term entry");
        return fail(LRH_ENOTHERM, "term " + std::to_string(t0) + " is not Hermitian");
    }
    return LRH_OK;
}

PassIO plain_io(const lrh_problem* p) {
    PassIO io{};
    io.nu_in = p->P.nu;
    io.zeta_in = p->opt.variant == LRH_NESTEROV ? p->P.zeta : nullptr;
    io.rho_out = p->P.rho;
    io.tr_out = p->P.tr;
    return io;
}

// Region pass of every size class: one launch for all classes (when chosen and possible), or
// class 0 on the problem's stream and the others on forked streams (independent work: disjoint
// outputs, read-only inputs; in a pending pass every updated message has exactly one owner),
// joined afterwards.  Only class 0 may be `writer`.
int launch_all_classes(lrh_problem* p, const PassIO& io0) {
    const size_t nc = p->class_k.size();
    if (p->fused && p->persist_grid > 0) {
        LRH_CK(launch_class_pass(p->P, p->plan, p->persist_kmax, io0, p->stream));
        return LRH_OK;
    }
    PassIO io = io0;
    io.writer = 0;
    if (!p->concurrent || nc < 2) {
        for (size_t c = 0; c < nc; ++c)
            LRH_CK(launch_region_pass(p->P, c == 0 ? io0 : io, p->class_k[c], p->class_list[c], p->class_count[c],
                                      p->stream, p->class_block[c]));
        return LRH_OK;
    }
    LRH_CK(cudaEventRecord(p->ev_fork, p->stream));
    for (size_t c = 1; c < nc; ++c) {
        LRH_CK(cudaStreamWaitEvent(p->aux[c - 1], p->ev_fork, 0));
        LRH_CK(launch_region_pass(p->P, io, p->class_k[c], p->class_list[c], p->class_count[c], p->aux[c - 1],
                                  p->class_block[c]));
        LRH_CK(cudaEventRecord(p->ev_join[c - 1], p->aux[c - 1]));
    }
    LRH_CK(launch_region_pass(p->P, io0, p->class_k[0], p->class_list[0], p->class_count[0], p->stream, p->class_block[0]));
    for (size_t c = 1; c < nc; ++c) LRH_CK(cudaStreamWaitEvent(p->stream, p->ev_join[c - 1], 0));
    return LRH_OK;
}

// After n fused Alg. 2 passes: apply the pending update of the last pass (its multipliers in
// A when n = 1 or n - 1 is even, else B; its states in X when n - 1 is even, else Y) into the
// canonical A, and advance t0 by n.
int enqueue_nesterov_tail(lrh_problem* p, int n) {
    DevProblem& P = p->P;
    PassIO fin{};
    fin.rel = n - 1;
    fin.nu_in = (n == 1) ? P.nu : ((n - 1) % 2 == 1 ? P.nu_b : P.nu);
    fin.zeta_in = (n == 1) ? P.zeta : ((n - 1) % 2 == 1 ? P.zeta_b : P.zeta);
    fin.rho_in = ((n - 1) % 2 == 0) ? P.rho : P.rho_b;
    fin.tr_in = ((n - 1) % 2 == 0) ? P.tr : P.tr_b;
    fin.nu_out = P.nu;
    fin.zeta_out = P.zeta;
    LRH_CK(launch_finalize(P, fin, p->stream));
    LRH_CK(launch_advance(P, n, p->stream));
    return LRH_OK;
}

// Driver lrh_step uses now (LRH_LOOP_EAGER / GRAPH / PERSISTENT).
int effective_loop(const lrh_problem* p) {
    int m = p->opt.loop;
    if (m == LRH_LOOP_AUTO) m = p->loop_auto >= 0 ? p->loop_auto : LRH_LOOP_GRAPH;
    if (m == LRH_LOOP_PERSISTENT && p->persist_grid <= 0) m = LRH_LOOP_GRAPH;
    return m;
}

// n iterations in one cooperative launch (plus, for Alg. 2, the finalisation of the last pass).
// Launches are split so that one launch's barrier arrivals (grid x barriers) stay below 2^30:
// the 32-bit arrival counter never wraps.  Split Alg. 2 steps are bit-identical to one step.
int run_persistent(lrh_problem* p, int n) {
    PersistPlan L = p->plan;
    L.nesterov = p->opt.variant == LRH_NESTEROV ? 1 : 0;
    const int64_t per_iter = L.nesterov ? 1 : 3;
    const int64_t max_n = std::max<int64_t>(1, ((int64_t)1 << 30) / ((int64_t)p->persist_grid * per_iter));
    for (int done = 0; done < n;) {
        const int c = (int)std::min<int64_t>(max_n, n - done);
        L.n = c;
        L.par0 = (int)((p->iteration + done) & 1);
        LRH_CK(launch_persistent(p->P, L, p->persist_kmax, p->persist_grid, p->stream));
        if (L.nesterov) {
            const int rc = enqueue_nesterov_tail(p, c);
            if (rc) return rc;
        }
        done += c;
    }
    return LRH_OK;
}

// Classes of 3 and 4 sites whose launch shape selects the 2x2-block layout (bit k).
int32_t blk_mask_of(const lrh_problem* p) {
    int32_t m = 0;
    for (size_t c = 0; c < p->class_k.size(); ++c) {
        if ((p->class_k[c] == 3 || p->class_k[c] == 4) && p->class_block[c] > LRH_SHAPE_BLOCKS) m |= 1 << p->class_k[c];
        if (p->class_k[c] == 4 && p->class_block[c] > LRH_SHAPE_WARP16) m |= 1 << 5;
    }
    return m;
}

// Tiles of the persistent / one-launch pass for the current launch shapes: classes in cost order
// (heaviest first), persistent_tile_regions(k, layout) regions per tile, grid = min(tiles,
// resident CTAs).  Called at creation and whenever a launch shape changes.
void layout_plan(lrh_problem* p) {
    if (p->persist_cap <= 0) return;
    PersistPlan& L = p->plan;
    L.blk_mask = blk_mask_of(p);
    int64_t tiles = 0;
    for (size_t c = 0; c < p->class_k.size(); ++c) {
        const int64_t per = persistent_tile_regions(p->class_k[c], L.blk_mask);
        L.cls[c] = p->class_list[c];
        L.count[c] = p->class_count[c];
        L.k[c] = p->class_k[c];
        L.tile0[c] = tiles;
        tiles += ((int64_t)p->n_inst * p->class_count[c] + per - 1) / per;
    }
    L.tiles = tiles;
    L.n_classes = (int32_t)p->class_k.size();
    p->persist_grid = (int)std::min<int64_t>(tiles, p->persist_cap);
}

// The persistent launch's barrier word and resident-CTA capacity.  Not available when a class has
// more than 4 sites or the device lacks cooperative launches.
int plan_persistent(lrh_problem* p) {
    p->persist_grid = 0;
    p->persist_cap = 0;
    const size_t nc = p->class_k.size();
    if (nc == 0 || nc > (size_t)kPersistClasses) return LRH_OK;
    int kmax = 2;
    for (int k : p->class_k) { if (k > 4) return LRH_OK; kmax = std::max(kmax, k); }
    int coop = 0, sms = 0, nb = 0;
    LRH_CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, p->device));
    LRH_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
    if (!coop) return LRH_OK;
    LRH_CK(persistent_prepare(kmax, &nb));
    if (nb <= 0) return LRH_OK;
    PersistPlan L{};
    int rc;
    if ((rc = p->dalloc(&L.bar, 2))) return rc;
    LRH_CK(cudaMemset(L.bar, 0, 2 * sizeof(unsigned)));
    p->plan = L;
    p->persist_kmax = kmax;
    p->persist_cap = (int64_t)nb * sms;
    layout_plan(p);
    return LRH_OK;
}

// Alg. 2, n iterations as n region passes: pass 0 reads the canonical nu, zeta; pass j >= 1
// first applies iteration j-1's pending update (owners write it to the other buffer:
// odd j -> B, even j -> A) and writes its states to X (even j) or Y (odd j); then the
// pending update of the last pass is written into the canonical A, and t0 advances by n.
int enqueue_nesterov(lrh_problem* p, int n) {
    DevProblem& P = p->P;
    float2* nuA = P.nu; float2* zA = P.zeta; float2* nuB = P.nu_b; float2* zB = P.zeta_b;
    float2* rX = P.rho; float2* tX = P.tr; float2* rY = P.rho_b; float2* tY = P.tr_b;
    PassIO io{};
    for (int j = 0; j < n; ++j) {
        io = PassIO{};
        io.rel = j;
        io.writer = 1;
        io.pending = j > 0;
        io.nu_in = (j % 2 == 1 || j == 0) ? nuA : nuB;
        io.zeta_in = (j % 2 == 1 || j == 0) ? zA : zB;
        if (j > 0) {
            io.rho_in = (j % 2 == 1) ? rX : rY;
            io.tr_in = (j % 2 == 1) ? tX : tY;
            io.nu_out = (j % 2 == 1) ? nuB : nuA;
            io.zeta_out = (j % 2 == 1) ? zB : zA;
        }
        io.rho_out = (j % 2 == 0) ? rX : rY;
        io.tr_out = (j % 2 == 0) ? tX : tY;
        int rc = launch_all_classes(p, io);
        if (rc) return rc;
    }
    return enqueue_nesterov_tail(p, n);
}

void drop_graphs(lrh_problem* p) {
    if (p->graph_exec) { cudaGraphExecDestroy(p->graph_exec); p->graph_exec = nullptr; }
    if (p->graph) { cudaGraphDestroy(p->graph); p->graph = nullptr; }
    for (auto& g : p->nest_graphs) cudaGraphExecDestroy(g.second);
    p->nest_graphs.clear();
}

int step_nesterov(lrh_problem* p, int n) {
    if (n <= 0) return LRH_OK;
    const int mode = effective_loop(p);
    if (mode == LRH_LOOP_PERSISTENT) return run_persistent(p, n);
    if (mode == LRH_LOOP_EAGER || n < 2) return enqueue_nesterov(p, n);
    cudaGraphExec_t ge = nullptr;
    for (auto& g : p->nest_graphs) if (g.first == n) ge = g.second;
    if (!ge) {
        LRH_CK(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_nesterov(p, n);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(p->stream, &g);
        if (rc != LRH_OK) { if (g) cudaGraphDestroy(g); return rc; }
        if (e != cudaSuccess) return fail(LRH_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(LRH_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
        if (p->nest_graphs.size() >= 8) { cudaGraphExecDestroy(p->nest_graphs.front().second); p->nest_graphs.erase(p->nest_graphs.begin()); }
        p->nest_graphs.emplace_back(n, ge);
    }
    LRH_CK(cudaGraphLaunch(ge, p->stream));
    return LRH_OK;
}

int run_iteration(lrh_problem* p, int par) {
    int rc = launch_all_classes(p, plain_io(p));
    if (rc) return rc;
    if (p->opt.variant == LRH_SUBGRADIENT) LRH_CK(launch_reduce(p->P, p->P.val, 1, p->stream));
    LRH_CK(launch_update(p->P, par, UPD_STEP, p->stream));
    return LRH_OK;
}

int build_graph(lrh_problem* p) {
    LRH_CK(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
    int rc = LRH_OK;
    for (int i = 0; i < kGraphChunk && rc == LRH_OK; ++i) rc = run_iteration(p, i & 1);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(p->stream, &g);
    if (rc != LRH_OK) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return fail(LRH_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    p->graph = g;
    LRH_CK(cudaGraphInstantiate(&p->graph_exec, g, 0));
    return LRH_OK;
}

// Wait for the stream and report the device error word; every reported condition is cleared,
// so it is returned once, by the first synchronising call after it was raised.
int read_err(lrh_problem* p) {
    int32_t h = 0;
    LRH_CK(cudaMemcpyAsync(&h, p->P.err, sizeof(int32_t), cudaMemcpyDeviceToHost, p->stream));
    LRH_CK(cudaStreamSynchronize(p->stream));
    if (h) {
        LRH_CK(cudaMemsetAsync(p->P.err, 0, sizeof(int32_t), p->stream));
        LRH_CK(cudaStreamSynchronize(p->stream));
    }
    if (h & DEV_ERR_TIMEOUT)
        return fail(LRH_ETIMEOUT, "a bounded device wait (grid barrier of the persistent iteration, or a "
                                  "tensor-core commit) gave up; the results of that launch are incomplete");
    if (h & DEV_ERR_NUMERIC) return fail(LRH_ENUMERIC, "a non-finite eigenvalue, value or message was produced");
    if (h & DEV_ERR_NOCONV)
        return fail(LRH_ENOCONV, "an FP64 certification eigensolve stopped at its sweep cap; the bound is "
                                 "Weyl-corrected (still a lower bound) but looser");
    return LRH_OK;
}

// Host plan of a region family (no device work): validated regions, pairs (explicit, or the
// covering relation of inclusion), term placement (explicit, or the smallest containing region
// with the lowest index), and the constants Lambda_G, Gamma_G, kappa_G of the parameter rules.
struct PosetPlan {
    std::vector<std::vector<int32_t>> regs;
    std::vector<std::vector<std::pair<int, int>>> kids;   // per parent: (child, index-bit mask), ascending child
    int maxk = 0;
    std::vector<int32_t> place;       // term -> region
    std::vector<int32_t> term_mask;   // bits of the region's basis index that carry the term's sites
    double lambda_G = 0, gamma_G = 0;
    int32_t kappa = 0;
    int64_t n_pairs = 0;
};

int plan_poset(const lrh_problem_desc* d, PosetPlan& pl) {
    if (d->n_sites <= 0 || d->n_regions <= 0 || d->n_instances <= 0 || d->n_terms < 0)
        return fail(LRH_EINVAL, "n_sites, n_regions, n_instances must be positive");
    if (!d->region_ptr || !d->region_sites) return fail(LRH_EINVAL, "region arrays are NULL");
    if (d->n_terms > 0 && (!d->term_ptr || !d->term_sites || !d->term_mat_off))
        return fail(LRH_EINVAL, "term arrays are NULL");
    const int R = d->n_regions;
    auto& regs = pl.regs;
    auto& kids = pl.kids;
    regs.assign(R, {});
    kids.assign(R, {});
    std::unordered_map<std::vector<int32_t>, int, VecHash> index;
    index.reserve((size_t)R * 2);
    int maxk = 0;
    for (int e = 0; e < R; ++e) {
        const int64_t b = d->region_ptr[e], en = d->region_ptr[e + 1];
        const int64_t k = en - b;
        if (k < 1 || k > kMaxSites) return fail(LRH_EINVAL, "region " + std::to_string(e) + " has " + std::to_string(k) + " sites (1..8 allowed)");
        regs[e].assign(d->region_sites + b, d->region_sites + en);
        for (int64_t i = 0; i < k; ++i) {
            if (regs[e][i] < 0 || regs[e][i] >= d->n_sites) return fail(LRH_EINVAL, "region site out of range");
            if (i && regs[e][i] <= regs[e][i - 1]) return fail(LRH_EINVAL, "region sites must be sorted and unique");
        }
        if (!index.emplace(regs[e], e).second) return fail(LRH_EPOSET, "duplicate region " + std::to_string(e));
        maxk = std::max<int>(maxk, (int)k);
    }
    pl.maxk = maxk;
    if (d->n_pairs < 0) return fail(LRH_EINVAL, "n_pairs < 0");
    if (d->n_pairs > 0) {
        // explicit pairs: the child's sites must be a proper subset of the parent's
        if (!d->pair_parent || !d->pair_child) return fail(LRH_EINVAL, "pair arrays are NULL");
        std::set<std::pair<int, int>> seen;
        for (int64_t q = 0; q < d->n_pairs; ++q) {
            const int e = d->pair_parent[q], f = d->pair_child[q];
            if (e < 0 || e >= R || f < 0 || f >= R) return fail(LRH_EINVAL, "pair region index out of range");
            if (!seen.insert({e, f}).second) return fail(LRH_EPOSET, "duplicate pair " + std::to_string(e) + "->" + std::to_string(f));
            const int k = (int)regs[e].size();
            if (regs[f].size() >= regs[e].size()) return fail(LRH_EPOSET, "pair child is not a proper subset of its parent");
            int im = 0;
            for (int32_t site : regs[f]) {
                const auto it = std::find(regs[e].begin(), regs[e].end(), site);
                if (it == regs[e].end()) return fail(LRH_EPOSET, "pair child is not a subset of its parent");
                im |= 1 << (k - 1 - (int)(it - regs[e].begin()));
            }
            kids[e].emplace_back(f, im);
        }
        for (auto& v : kids) std::sort(v.begin(), v.end());
    }
    // covering pairs (children of e: proper sub-regions with no region strictly between)
    for (int e = 0; e < R && d->n_pairs == 0; ++e) {
        const int k = (int)regs[e].size();
        std::vector<std::pair<int, int>> subs;   // (region, position mask: bit p = position p)
        std::vector<int32_t> tmp;
        for (int m = 1; m < (1 << k) - 1; ++m) {
            tmp.clear();
            for (int p = 0; p < k; ++p) if (m >> p & 1) tmp.push_back(regs[e][p]);
            auto it = index.find(tmp);
            if (it != index.end()) subs.emplace_back(it->second, m);
        }
        for (auto& f : subs) {
            bool covered = true;
            for (auto& gq : subs)
                if (gq.second != f.second && (f.second & gq.second) == f.second) { covered = false; break; }
            if (!covered) continue;
            int im = 0;
            for (int p = 0; p < k; ++p) if (f.second >> p & 1) im |= 1 << (k - 1 - p);
            kids[e].emplace_back(f.first, im);
        }
        std::sort(kids[e].begin(), kids[e].end());
    }
    // Lambda_G, Gamma_G and kappa_G
    std::vector<int64_t> n_par(R, 0);
    pl.n_pairs = 0;
    for (int e = 0; e < R; ++e) for (auto& f : kids[e]) { ++n_par[f.first]; ++pl.n_pairs; }
    bool level1 = maxk <= 2;
    for (int e = 0; e < R; ++e) for (auto& f : kids[e]) if (!(regs[e].size() == 2 && regs[f.first].size() == 1)) level1 = false;
    if (level1) {
        int64_t deg = 0;
        for (int e = 0; e < R; ++e) deg = std::max(deg, n_par[e]);
        pl.lambda_G = (double)deg + 2.0;
    } else {
        double best = 0;
        for (int e = 0; e < R; ++e)
            for (auto& f : kids[e]) {
                const double me = (double)(n_par[e] + (int64_t)kids[e].size());
                const double mf = (double)(n_par[f.first] + (int64_t)kids[f.first].size());
                const double ratio = std::ldexp(1.0, (int)regs[e].size() - (int)regs[f.first].size());
                best = std::max(best, mf + me * ratio);
            }
        pl.lambda_G = best;
    }
    pl.gamma_G = 0;
    for (int e = 0; e < R; ++e) pl.gamma_G += (double)regs[e].size() * std::log(2.0);
    {   // kappa_G = max over sites i of |{e->f : i in f}| (Thm 6)
        std::vector<int32_t> cnt(d->n_sites, 0);
        for (int e = 0; e < R; ++e) for (auto& f : kids[e]) for (int32_t site : regs[f.first]) ++cnt[site];
        pl.kappa = cnt.empty() ? 0 : *std::max_element(cnt.begin(), cnt.end());
    }
    // term placement
    std::vector<std::vector<int32_t>> by_site(d->n_sites);
    for (int e = 0; e < R; ++e) for (int32_t s : regs[e]) by_site[s].push_back(e);
    pl.place.assign(d->n_terms, -1);
    pl.term_mask.assign(d->n_terms, 0);
    for (int t = 0; t < d->n_terms; ++t) {
        const int64_t b = d->term_ptr[t], en = d->term_ptr[t + 1];
        if (en - b < 1 || en - b > kMaxSites) return fail(LRH_EINVAL, "term " + std::to_string(t) + " has a bad site count");
        std::vector<int32_t> ts(d->term_sites + b, d->term_sites + en);
        for (size_t i = 0; i < ts.size(); ++i) {
            if (ts[i] < 0 || ts[i] >= d->n_sites) return fail(LRH_EINVAL, "term site out of range");
            if (i && ts[i] <= ts[i - 1]) return fail(LRH_EINVAL, "term sites must be sorted and unique");
        }
        int bestr = -1;
        if (d->term_region) {
            bestr = d->term_region[t];
            if (bestr < 0 || bestr >= R) return fail(LRH_EINVAL, "term_region out of range");
            if (!std::includes(regs[bestr].begin(), regs[bestr].end(), ts.begin(), ts.end()))
                return fail(LRH_EPOSET, "term " + std::to_string(t) + " does not fit in its term_region");
        } else {
            for (int32_t e : by_site[ts[0]]) {
                if (!std::includes(regs[e].begin(), regs[e].end(), ts.begin(), ts.end())) continue;
                if (bestr < 0 || regs[e].size() < regs[bestr].size() || (regs[e].size() == regs[bestr].size() && e < bestr)) bestr = e;
            }
            if (bestr < 0) return fail(LRH_EPOSET, "term " + std::to_string(t) + " fits in no region");
        }
        const int64_t Dt = (int64_t)1 << ts.size();
        const int64_t off = d->term_mat_off[t];
        if (off < 0 || off + Dt * Dt > d->term_mat_total) return fail(LRH_EINVAL, "term matrix offset out of range");
        const int k = (int)regs[bestr].size();
        int M = 0;
        for (int32_t site : ts) {
            const int pos = (int)(std::find(regs[bestr].begin(), regs[bestr].end(), site) - regs[bestr].begin());
            M |= 1 << (k - 1 - pos);
        }
        pl.place[t] = bestr;
        pl.term_mask[t] = M;
    }
    return LRH_OK;
}

}  // namespace

extern "C" {

const char* lrh_strerror(int code) {
    switch (code) {
        case LRH_OK: return "ok";
        case LRH_EINVAL: return "invalid argument";
        case LRH_ENOTHERM: return "term matrix is not Hermitian";
        case LRH_EPOSET: return "invalid region family";
        case LRH_ENOMEM: return "out of memory";
        case LRH_ECUDA: return "CUDA error";
        case LRH_ETIMEOUT: return "device wait timed out";
        case LRH_ENUMERIC: return "non-finite value";
        case LRH_EUNSUPPORTED: return "unsupported region size";
        case LRH_ENOCONV: return "certification eigensolve not converged (bound still valid)";
        case LRH_EDEADLINE: return "deadline reached";
        default: return "unknown error";
    }
}

const char* lrh_last_error(void) { return g_last_error.c_str(); }

int lrh_create(const lrh_problem_desc* d, const lrh_options* opts, void* stream, lrh_problem** out) {
    if (!out) return fail(LRH_EINVAL, "out is NULL");
    *out = nullptr;
    if (!d) return fail(LRH_EINVAL, "desc is NULL");
    int rc = validate_options(opts);
    if (rc) return rc;
    if (d->n_sites <= 0 || d->n_regions <= 0 || d->n_instances <= 0 || d->n_terms < 0)
        return fail(LRH_EINVAL, "n_sites, n_regions, n_instances must be positive");
    if (!d->region_ptr || !d->region_sites) return fail(LRH_EINVAL, "region arrays are NULL");
    if (d->n_terms > 0 && (!d->term_ptr || !d->term_sites || !d->term_mat_off || !d->term_mats))
        return fail(LRH_EINVAL, "term arrays are NULL");

    PosetPlan pl;
    if ((rc = plan_poset(d, pl))) return rc;
    const int R = d->n_regions;
    const auto& regs = pl.regs;
    const auto& kids = pl.kids;
    const int maxk = pl.maxk;
    if (maxk > kMaxKernelSites)
        return fail(LRH_EUNSUPPORTED, "regions of " + std::to_string(maxk) + " sites have no region-pass kernel in this build (at most " +
                                          std::to_string(kMaxKernelSites) + ")");
    lrh_problem* p = new (std::nothrow) lrh_problem();
    if (!p) return fail(LRH_ENOMEM, "host allocation");
    std::unique_ptr<lrh_problem> guard(p);
    p->n_sites = d->n_sites;
    p->n_inst = d->n_instances;
    copy_options(p, opts);
    p->n_regions = R;
    p->max_k = maxk;
    cudaGetDevice(&p->device);
    p->ghost.assign(R, 0);
    if (d->region_ghost)
        for (int e = 0; e < R; ++e) p->ghost[e] = d->region_ghost[e] ? 1 : 0;
    p->has_ghost = std::find(p->ghost.begin(), p->ghost.end(), 1) != p->ghost.end();
    if (std::find(p->ghost.begin(), p->ghost.end(), 0) == p->ghost.end())
        return fail(LRH_EINVAL, "every region is a ghost region");

    std::vector<PairInfo> pairs;
    std::vector<std::vector<int32_t>> parent_of(R);
    std::vector<RegionInfo> rinfo(R);
    std::vector<int32_t> child_pairs, parent_pairs;
    int64_t moff = 0;
    for (int e = 0; e < R; ++e) {
        rinfo[e].child_begin = (int32_t)child_pairs.size();
        for (auto& f : kids[e]) {
            PairInfo pi;
            pi.off = moff;
            pi.parent = e;
            pi.child = f.first;
            pi.mask = f.second;
            pi.kf = (int32_t)regs[f.first].size();
            moff += (int64_t)1 << (2 * pi.kf);
            parent_of[f.first].push_back((int32_t)pairs.size());
            child_pairs.push_back((int32_t)pairs.size());
            pairs.push_back(pi);
        }
        rinfo[e].child_end = (int32_t)child_pairs.size();
    }
    for (int e = 0; e < R; ++e) {
        rinfo[e].parent_begin = (int32_t)parent_pairs.size();
        for (int32_t q : parent_of[e]) parent_pairs.push_back(q);
        rinfo[e].parent_end = (int32_t)parent_pairs.size();
    }
    p->n_pairs = (int32_t)pairs.size();
    p->msg_elems = moff;
    for (auto& pi : pairs) { p->pair_parent.push_back(pi.parent); p->pair_child.push_back(pi.child); p->pair_off.push_back(pi.off); }
    p->lambda_G = pl.lambda_G;
    p->gamma_G = pl.gamma_G;
    p->kappa = pl.kappa;

    // ---------------------------------------------------------------- terms
    std::vector<char> has_term(R, 0);
    p->n_terms = d->n_terms;
    p->term_total = d->term_mat_total;
    for (int t = 0; t < d->n_terms; ++t) {
        has_term[pl.place[t]] = 1;
        p->term_region.push_back(pl.place[t]);
        p->term_mask.push_back(pl.term_mask[t]);
        p->term_kt.push_back((int32_t)(d->term_ptr[t + 1] - d->term_ptr[t]));
        p->term_off.push_back(d->term_mat_off[t]);
    }
    if (d->n_terms > 0 && (rc = check_terms(p, d->term_ptr, d->term_mats))) return rc;
    int64_t hoff = 0, roff = 0, aoff = 0;
    p->region_h_off.assign(R, -1);
    p->region_k.assign(R, 0);
    for (int e = 0; e < R; ++e) {
        const int64_t D = (int64_t)1 << regs[e].size();
        p->region_k[e] = (int32_t)regs[e].size();
        rinfo[e].h_off = has_term[e] ? hoff : -1;
        p->region_h_off[e] = rinfo[e].h_off;
        if (has_term[e]) hoff += D * D;
        rinfo[e].rho_off = parent_of[e].empty() ? -1 : roff;
        if (!parent_of[e].empty()) roff += D * D;
        rinfo[e].all_off = aoff;
        aoff += D * D;
    }
    p->h_elems = hoff;
    p->rho_elems = roff;
    p->all_elems = aoff;
    for (auto& pi : pairs) pi.child_rho = rinfo[pi.child].rho_off;
    std::vector<double> h64;
    embed_terms(p, d->term_mats, h64);

    // ---------------------------------------------------------------- device state
    LRH_CK(prepare_kernels());
    LRH_CK(prepare_vjp_kernels());
    if (stream) {
        p->stream = (cudaStream_t)stream;
    } else {
        LRH_CK(cudaStreamCreate(&p->stream));   // blocking stream: ordered with the legacy default stream
        p->own_stream = true;
    }
    DevProblem& P = p->P;
    P.n_inst = p->n_inst;
    P.n_regions = R;
    P.n_pairs = p->n_pairs;
    P.h_elems = hoff;
    P.rho_elems = roff;
    P.msg_elems = moff;
    const int64_t NI = p->n_inst;
    RegionInfo* dreg; PairInfo* dpair; int32_t *dcp, *dpp, *dchunk;
    if ((rc = p->dalloc(&dreg, R)) || (rc = p->dalloc(&dpair, p->n_pairs)) || (rc = p->dalloc(&dcp, p->n_pairs)) ||
        (rc = p->dalloc(&dpp, p->n_pairs)) || (rc = p->dalloc(&dchunk, moff / 4)))
        return rc;
    {
        std::vector<int32_t> chunk((size_t)(moff / 4));
        for (size_t q = 0; q < pairs.size(); ++q) {
            const int64_t n4 = ((int64_t)1 << (2 * pairs[q].kf)) / 4;
            for (int64_t c = 0; c < n4; ++c) chunk[(size_t)(pairs[q].off / 4 + c)] = (int32_t)q;
        }
        if (!chunk.empty())
            LRH_CK(cudaMemcpy(dchunk, chunk.data(), sizeof(int32_t) * chunk.size(), cudaMemcpyHostToDevice));
    }
    P.chunk_pair = dchunk;
    {
        std::vector<int64_t> crho((size_t)std::max<int64_t>(moff / 4, 1));
        for (size_t q = 0; q < pairs.size(); ++q) {
            const int64_t n4 = ((int64_t)1 << (2 * pairs[q].kf)) / 4;
            for (int64_t c = 0; c < n4; ++c) crho[(size_t)(pairs[q].off / 4 + c)] = rinfo[pairs[q].child].rho_off - pairs[q].off;
        }
        std::vector<PairInfo> cinfo, pinfo;
        for (int32_t q : child_pairs) cinfo.push_back(pairs[q]);
        for (int32_t q : parent_pairs) pinfo.push_back(pairs[q]);
        int64_t* dcr; PairInfo *dci, *dpi;
        if ((rc = p->dalloc(&dcr, (int64_t)crho.size())) || (rc = p->dalloc(&dci, (int64_t)cinfo.size())) ||
            (rc = p->dalloc(&dpi, (int64_t)pinfo.size())))
            return rc;
        LRH_CK(cudaMemcpy(dcr, crho.data(), sizeof(int64_t) * crho.size(), cudaMemcpyHostToDevice));
        if (!cinfo.empty()) LRH_CK(cudaMemcpy(dci, cinfo.data(), sizeof(PairInfo) * cinfo.size(), cudaMemcpyHostToDevice));
        if (!pinfo.empty()) LRH_CK(cudaMemcpy(dpi, pinfo.data(), sizeof(PairInfo) * pinfo.size(), cudaMemcpyHostToDevice));
        P.chunk_rho = dcr;
        P.child_info = dci;
        P.parent_info = dpi;
    }
    float2* h32; double2* dh64;
    if ((rc = p->dalloc(&h32, NI * hoff)) || (rc = p->dalloc(&dh64, NI * hoff))) return rc;
    if ((rc = p->dalloc(&P.nu, NI * moff)) || (rc = p->dalloc(&P.zeta, NI * moff)) || (rc = p->dalloc(&P.nu_best, NI * moff)) ||
        (rc = p->dalloc(&P.tr, NI * moff)) || (rc = p->dalloc(&P.grad, NI * moff)) || (rc = p->dalloc(&P.rho, NI * roff)))
        return rc;
    if (p->opt.variant == LRH_NESTEROV || true) {
        if ((rc = p->dalloc(&P.nu_b, NI * moff)) || (rc = p->dalloc(&P.zeta_b, NI * moff)) ||
            (rc = p->dalloc(&P.rho_b, NI * roff)) || (rc = p->dalloc(&P.tr_b, NI * moff)))
            return rc;
    }
    if ((rc = p->dalloc(&P.val, NI * R)) || (rc = p->dalloc(&P.val64, NI * R)) || (rc = p->dalloc(&P.q_sum, NI)) ||
        (rc = p->dalloc(&P.q_best, NI)) || (rc = p->dalloc(&P.best_flag, NI)) || (rc = p->dalloc(&P.st, 1)) ||
        (rc = p->dalloc(&P.err, 1)) || (rc = p->dalloc(&P.sweeps, kClassSlots)) || (rc = p->dalloc(&P.capped, kClassSlots)))
        return rc;
    P.reg = dreg; P.pair = dpair; P.child_pairs = dcp; P.parent_pairs = dpp; P.h32 = h32; P.h64 = dh64;
    P.all_elems = p->all_elems;
    P.n_terms = p->n_terms;
    P.term_total = p->term_total;
    LRH_CK(cudaMemcpy(dreg, rinfo.data(), sizeof(RegionInfo) * R, cudaMemcpyHostToDevice));
    if (p->n_pairs) {
        LRH_CK(cudaMemcpy(dpair, pairs.data(), sizeof(PairInfo) * pairs.size(), cudaMemcpyHostToDevice));
        LRH_CK(cudaMemcpy(dcp, child_pairs.data(), sizeof(int32_t) * child_pairs.size(), cudaMemcpyHostToDevice));
        LRH_CK(cudaMemcpy(dpp, parent_pairs.data(), sizeof(int32_t) * parent_pairs.size(), cudaMemcpyHostToDevice));
    }
    if ((rc = upload_terms(p, h64))) return rc;
    LRH_CK(cudaMemset(P.nu, 0, sizeof(float2) * std::max<int64_t>(NI * moff, 1)));
    LRH_CK(cudaMemset(P.zeta, 0, sizeof(float2) * std::max<int64_t>(NI * moff, 1)));
    LRH_CK(cudaMemset(P.nu_best, 0, sizeof(float2) * std::max<int64_t>(NI * moff, 1)));
    LRH_CK(cudaMemset(P.grad, 0, sizeof(float2) * std::max<int64_t>(NI * moff, 1)));
    LRH_CK(cudaMemset(P.best_flag, 0, sizeof(int32_t) * NI));
    LRH_CK(cudaMemset(P.err, 0, sizeof(int32_t)));
    LRH_CK(cudaMemset(P.sweeps, 0, sizeof(unsigned long long) * kClassSlots));
    LRH_CK(cudaMemset(P.capped, 0, sizeof(unsigned long long) * kClassSlots));
    LRH_CK(cudaMemset(P.val64, 0, sizeof(double) * NI * R));
    LRH_CK(cudaMemset(P.val, 0, sizeof(double) * NI * R));
    LRH_CK(cudaMemset(P.st, 0, sizeof(IterState)));
    {
        std::vector<double> ninf(NI, -std::numeric_limits<double>::infinity());
        LRH_CK(cudaMemcpy(P.q_best, ninf.data(), sizeof(double) * NI, cudaMemcpyHostToDevice));
    }
    // size classes
    for (int k = 0; k < kClassSlots; ++k) P.class_base[k] = -1;
    P.class_uniform = 0;
    for (int k = 1; k <= kMaxSites; ++k) {
        std::vector<int32_t> lst;
        for (int e = 0; e < R; ++e) if ((int)regs[e].size() == k && !p->ghost[e]) lst.push_back(e);   // ghosts: no pass here
        if (lst.empty()) continue;
        int32_t* dl;
        if ((rc = p->dalloc(&dl, (int64_t)lst.size()))) return rc;
        LRH_CK(cudaMemcpy(dl, lst.data(), sizeof(int32_t) * lst.size(), cudaMemcpyHostToDevice));
        p->class_k.push_back(k);
        p->class_count.push_back((int32_t)lst.size());
        p->class_list.push_back(dl);
        bool contiguous = true;
        for (size_t i = 1; i < lst.size(); ++i) contiguous = contiguous && lst[i] == lst[0] + (int32_t)i;
        P.class_base[k] = contiguous ? lst[0] : -1;
        // uniform class: every record is the first one shifted (checked field by field)
        bool uniform = contiguous;
        const int64_t D2 = (int64_t)1 << (2 * k);
        for (size_t i = 0; uniform && i < lst.size(); ++i) {
            const RegionInfo u = uniform_region(rinfo[lst[0]], (int64_t)i, D2);
            const RegionInfo& g = rinfo[lst[i]];
            uniform = u.h_off == g.h_off && u.rho_off == g.rho_off && u.child_begin == g.child_begin &&
                      u.child_end == g.child_end && u.parent_begin == g.parent_begin && u.parent_end == g.parent_end &&
                      u.all_off == g.all_off;
        }
        if (uniform) {
            P.class_first[k] = rinfo[lst[0]];
            P.class_uniform |= 1 << k;
        }
    }
    // most expensive class first (it stays on the problem's stream)
    {
        std::vector<size_t> order(p->class_k.size());
        for (size_t c = 0; c < order.size(); ++c) order[c] = c;
        std::sort(order.begin(), order.end(), [&](size_t a, size_t b) {
            const double ca = (double)p->class_count[a] * std::pow(8.0, p->class_k[a]);
            const double cb = (double)p->class_count[b] * std::pow(8.0, p->class_k[b]);
            return ca > cb;
        });
        std::vector<int> k2; std::vector<int32_t> c2; std::vector<int32_t*> l2;
        for (size_t c : order) { k2.push_back(p->class_k[c]); c2.push_back(p->class_count[c]); l2.push_back(p->class_list[c]); }
        p->class_k = k2; p->class_count = c2; p->class_list = l2;
    }
    p->class_block.assign(p->class_k.size(), 128);
    for (size_t c = 0; c < p->class_k.size(); ++c) {
        if (p->class_k[c] >= 6) p->class_block[c] = LRH_SHAPE_CTA_FP32;   // CTA classes: FP32 back-transform
        if (p->class_k[c] == 3 || p->class_k[c] == 4) p->class_block[c] = LRH_SHAPE_BLOCKS + 128;   // 2x2-block layout
    }
    p->P.tc_backtransform = 0;
    // stored eigenbases of the 2x2-block classes (regions of 3 and 4 sites) and of the CTA classes
    // of 6 and 7 sites, the identity at first (none for a problem created with cold starts)
    for (int k = 0; k < kClassSlots; ++k) P.warm_off[k] = -1;
    for (size_t c = 0; c < p->class_k.size() && !p->opt.cold_start; ++c) {
        const int k = p->class_k[c];
        if (k != 3 && k != 4 && k != 6 && k != 7) continue;
        P.warm_off[k] = p->warm_elems;
        p->warm_elems += NI * p->class_count[c] * ((int64_t)1 << (2 * k));
    }
    if (p->warm_elems > 0) {
        if ((rc = p->dalloc(&P.warm, p->warm_elems))) return rc;
        if ((rc = reset_warm(p))) return rc;
        LRH_CK(cudaStreamSynchronize(p->stream));
    }
    if (maxk == 8) {   // scratch slots of the D = 256 pass (theta overflow, V, rho, rotation log)
        int slots = 0;
        LRH_CK(big_launch_slots(&slots));
        const int64_t slot = big_slot_elems(kBigLogSweeps);
        if ((rc = p->dalloc(&P.big, (int64_t)slots * slot))) return rc;
        P.big_slot = slot;
        P.big_slots = slots;
        P.big_log_sweeps = kBigLogSweeps;
    }
    if ((rc = plan_persistent(p))) return rc;
    LRH_CK(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
    for (size_t c = 1; c < p->class_k.size(); ++c) {
        cudaStream_t a;
        cudaEvent_t e;
        LRH_CK(cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking));
        p->aux.push_back(a);
        LRH_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        p->ev_join.push_back(e);
    }
    p->h_pinned_len = std::max<int64_t>(NI * R, 16);
    LRH_CK(cudaMallocHost(&p->h_pinned, sizeof(double) * p->h_pinned_len));
    if ((rc = push_state(p, true, 1.0, 0.0))) return rc;
    LRH_CK(cudaStreamSynchronize(p->stream));
    *out = guard.release();
    return LRH_OK;
}

void lrh_destroy(lrh_problem* p) {
    if (!p) return;
    DeviceGuard dg(p->device);
    if (p->stream) cudaStreamSynchronize(p->stream);
    delete p;
}

int lrh_get_info(const lrh_problem* p, lrh_info* info) {
    if (!p || !info) return fail(LRH_EINVAL, "NULL argument");
    DeviceGuard dg(p->device);
    std::memset(info, 0, sizeof(*info));
    info->n_instances = p->n_inst;
    info->n_regions = p->n_regions;
    info->n_pairs = p->n_pairs;
    info->max_region_sites = p->max_k;
    info->msg_elems = p->msg_elems;
    info->lambda_G = p->lambda_G;
    info->gamma_G = p->gamma_G;
    info->iteration = p->iteration;
    info->n_classes = (int32_t)p->class_k.size();
    unsigned long long sw[kClassSlots] = {0}, cap[kClassSlots] = {0};
    LRH_CK(cudaMemcpyAsync(sw, p->P.sweeps, sizeof(sw), cudaMemcpyDeviceToHost, p->stream));
    LRH_CK(cudaMemcpyAsync(cap, p->P.capped, sizeof(cap), cudaMemcpyDeviceToHost, p->stream));
    LRH_CK(cudaStreamSynchronize(p->stream));
    for (size_t c = 0; c < p->class_k.size() && c < 8; ++c) {
        info->class_sites[c] = p->class_k[c];
        info->class_regions[c] = p->class_count[c];
        info->sweeps[c] = sw[p->class_k[c]];
        info->sweep_capped[c] = cap[p->class_k[c]];
        info->class_block[c] = p->class_block[c];
    }
    info->n_sites = p->n_sites;
    info->kappa_G = p->kappa;
    info->warm_bytes = (int64_t)sizeof(float2) * p->warm_elems;
    info->concurrent_classes = (p->fused && p->persist_grid > 0) ? 2 : (p->concurrent ? 1 : 0);
    info->loop = effective_loop(p);
    info->persistent_grid = p->persist_grid;
    info->persistent_tiles = p->persist_grid > 0 ? p->plan.tiles : 0;
    return LRH_OK;
}

int lrh_get_pairs(const lrh_problem* p, int32_t* parent, int32_t* child, int64_t* msg_off) {
    if (!p) return fail(LRH_EINVAL, "NULL problem");
    if (parent) std::copy(p->pair_parent.begin(), p->pair_parent.end(), parent);
    if (child) std::copy(p->pair_child.begin(), p->pair_child.end(), child);
    if (msg_off) std::copy(p->pair_off.begin(), p->pair_off.end(), msg_off);
    return LRH_OK;
}

int lrh_set_options(lrh_problem* p, const lrh_options* opts) {
    if (!p) return fail(LRH_EINVAL, "NULL problem");
    int rc = validate_options(opts);
    if (rc) return rc;
    DeviceGuard dg(p->device);
    copy_options(p, opts);
    return push_state(p, false, 0.0, 0.0);
}

int lrh_restart(lrh_problem* p) {
    if (!p) return fail(LRH_EINVAL, "NULL problem");
    DeviceGuard dg(p->device);
    int rc = push_state(p, true, 1.0, 0.0);
    if (rc) return rc;
    if (p->opt.variant == LRH_SUBGRADIENT) {   // a new Alg. 1 run: q_best = -inf
        std::vector<double> ninf(p->n_inst, -std::numeric_limits<double>::infinity());
        LRH_CK(cudaMemcpyAsync(p->P.q_best, ninf.data(), sizeof(double) * p->n_inst, cudaMemcpyHostToDevice, p->stream));
        LRH_CK(cudaMemsetAsync(p->P.best_flag, 0, sizeof(int32_t) * p->n_inst, p->stream));
        LRH_CK(cudaStreamSynchronize(p->stream));
    }
    LRH_CK(cudaMemcpyAsync(p->P.zeta, p->P.nu, sizeof(float2) * p->n_inst * p->msg_elems, cudaMemcpyDeviceToDevice, p->stream));
    return LRH_OK;
}

int lrh_step(lrh_problem* p, int32_t n_iters) {
    if (!p || n_iters < 0) return fail(LRH_EINVAL, "bad arguments to lrh_step");
    if (p->has_ghost) return fail(LRH_EUNSUPPORTED, "problems with ghost regions iterate with lrh_halo_pass / lrh_halo_update");
    DeviceGuard dg(p->device);
    int rc;
    if (p->opt.variant == LRH_NESTEROV) {
        if ((rc = step_nesterov(p, n_iters))) return rc;
        p->iteration += n_iters;
        return LRH_OK;
    }
    const int mode = effective_loop(p);
    if (mode == LRH_LOOP_PERSISTENT) {
        if ((rc = run_persistent(p, n_iters))) return rc;
        p->iteration += n_iters;
        return LRH_OK;
    }
    while (n_iters > 0) {
        if (mode == LRH_LOOP_GRAPH && (p->iteration & 1) == 0 && n_iters >= kGraphChunk) {
            if (!p->graph_exec && (rc = build_graph(p))) return rc;
            LRH_CK(cudaGraphLaunch(p->graph_exec, p->stream));
            p->iteration += kGraphChunk;
            n_iters -= kGraphChunk;
        } else {
            if ((rc = run_iteration(p, (int)(p->iteration & 1)))) return rc;
            p->iteration += 1;
            n_iters -= 1;
        }
    }
    return LRH_OK;
}

int lrh_evaluate(lrh_problem* p) {
    if (!p) return fail(LRH_EINVAL, "NULL problem");
    if (p->has_ghost) return fail(LRH_EUNSUPPORTED, "problems with ghost regions iterate with lrh_halo_pass / lrh_halo_update");
    DeviceGuard dg(p->device);
    const int par = (int)(p->iteration & 1);
    int rc = launch_all_classes(p, plain_io(p));
    if (rc) return rc;
    LRH_CK(launch_update(p->P, par, UPD_GRAD_ONLY, p->stream));
    return LRH_OK;
}

int lrh_launch_region_pass(lrh_problem* p, int32_t k_sites) {
    if (!p) return fail(LRH_EINVAL, "NULL problem");
    DeviceGuard dg(p->device);
    for (size_t c = 0; c < p->class_k.size(); ++c)
        if (p->class_k[c] == k_sites) {
            LRH_CK(launch_region_pass(p->P, plain_io(p), k_sites, p->class_list[c], p->class_count[c], p->stream,
                                      p->class_block[c]));
            return LRH_OK;
        }
    return fail(LRH_EINVAL, "no region class with " + std::to_string(k_sites) + " sites");
}

int lrh_bound(lrh_problem* p, int32_t kind, double* out) {
    if (!p || !out) return fail(LRH_EINVAL, "NULL argument");
    DeviceGuard dg(p->device);
    const int64_t NI = p->n_inst;
    if (kind == LRH_BOUND_CERTIFIED) {
        const float2* msg = p->opt.variant == LRH_SUBGRADIENT ? p->P.nu_best : p->P.nu;
        for (size_t c = 0; c < p->class_k.size(); ++c)
            LRH_CK(launch_certify(p->P, p->class_k[c], p->class_list[c], p->class_count[c], msg, p->stream));
        LRH_CK(launch_reduce(p->P, p->P.val64, 0, p->stream));
        LRH_CK(cudaMemcpyAsync(p->h_pinned, p->P.q_sum, sizeof(double) * NI, cudaMemcpyDeviceToHost, p->stream));
    } else if (kind == LRH_BOUND_LAST) {
        LRH_CK(launch_reduce(p->P, p->P.val, 0, p->stream));
        LRH_CK(cudaMemcpyAsync(p->h_pinned, p->P.q_sum, sizeof(double) * NI, cudaMemcpyDeviceToHost, p->stream));
    } else if (kind == LRH_BOUND_BEST) {
        LRH_CK(cudaMemcpyAsync(p->h_pinned, p->P.q_best, sizeof(double) * NI, cudaMemcpyDeviceToHost, p->stream));
    } else {
        return fail(LRH_EINVAL, "unknown bound kind");
    }
    int rc = read_err(p);
    if (rc && rc != LRH_ENOCONV) return rc;
    std::copy(p->h_pinned, p->h_pinned + NI, out);   // with LRH_ENOCONV: valid, looser bounds
    return rc;
}

int lrh_get_region_values(lrh_problem* p, int32_t kind, double* out) {
    if (!p || !out) return fail(LRH_EINVAL, "NULL argument");
    DeviceGuard dg(p->device);
    const double* src = kind == LRH_BOUND_CERTIFIED ? p->P.val64 : (kind == LRH_BOUND_LAST ? p->P.val : nullptr);
    if (!src) return fail(LRH_EINVAL, "kind must be LRH_BOUND_LAST or LRH_BOUND_CERTIFIED");
    LRH_CK(cudaMemcpyAsync(out, src, sizeof(double) * p->n_inst * p->n_regions, cudaMemcpyDeviceToHost, p->stream));
    return read_err(p);
}

static float2* msg_array(lrh_problem* p, int which) {
    switch (which) {
        case LRH_MSG_NU: return p->P.nu;
        case LRH_MSG_ZETA: return p->P.zeta;
        case LRH_MSG_NU_BEST: return p->P.nu_best;
        case LRH_MSG_GRAD: return p->P.grad;
        default: return nullptr;
    }
}

int lrh_get_messages(lrh_problem* p, int32_t which, void* dst, int64_t bytes, int32_t dst_is_device) {
    if (!p || !dst) return fail(LRH_EINVAL, "NULL argument");
    float2* src = msg_array(p, which);
    if (!src) return fail(LRH_EINVAL, "unknown message array");
    const int64_t need = (int64_t)sizeof(float2) * p->n_inst * p->msg_elems;
    if (bytes != need) return fail(LRH_EINVAL, "bytes must be n_instances * msg_elems * 8 = " + std::to_string(need));
    DeviceGuard dg(p->device);
    if (need == 0) return LRH_OK;
    LRH_CK(cudaMemcpyAsync(dst, src, (size_t)need, dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, p->stream));
    if (!dst_is_device) LRH_CK(cudaStreamSynchronize(p->stream));
    return LRH_OK;
}

int lrh_set_messages(lrh_problem* p, int32_t which, const void* src, int64_t bytes, int32_t src_is_device) {
    if (!p || !src) return fail(LRH_EINVAL, "NULL argument");
    if (which == LRH_MSG_GRAD) return fail(LRH_EINVAL, "the gradient array is read only");
    float2* dst = msg_array(p, which);
    if (!dst) return fail(LRH_EINVAL, "unknown message array");
    const int64_t need = (int64_t)sizeof(float2) * p->n_inst * p->msg_elems;
    if (bytes != need) return fail(LRH_EINVAL, "bytes must be n_instances * msg_elems * 8 = " + std::to_string(need));
    DeviceGuard dg(p->device);
    if (need == 0) return LRH_OK;
    LRH_CK(cudaMemcpyAsync(dst, src, (size_t)need, src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, p->stream));
    if (!src_is_device) LRH_CK(cudaStreamSynchronize(p->stream));
    return LRH_OK;
}

int lrh_set_terms(lrh_problem* p, const double* term_mats) {
    if (!p || (!term_mats && p->n_terms > 0)) return fail(LRH_EINVAL, "NULL argument");
    DeviceGuard dg(p->device);
    std::vector<int64_t> tptr(p->n_terms + 1, 0);
    for (int t = 0; t < p->n_terms; ++t) tptr[t + 1] = tptr[t] + p->term_kt[t];
    int rc = check_terms(p, tptr.data(), term_mats);
    if (rc) return rc;
    std::vector<double> h64;
    embed_terms(p, term_mats, h64);
    LRH_CK(cudaStreamSynchronize(p->stream));
    return upload_terms(p, h64);
}

int lrh_vjp(lrh_problem* p, const double* q_bar, const void* g_bar, int32_t g_bar_is_device, void* nu_bar,
            void* term_bar, int32_t out_is_device) {
    if (!p || !q_bar) return fail(LRH_EINVAL, "NULL argument");
    if (p->has_ghost) return fail(LRH_EUNSUPPORTED, "problems with ghost regions iterate with lrh_halo_pass / lrh_halo_update");
    if (p->opt.variant != LRH_NESTEROV) return fail(LRH_EINVAL, "lrh_vjp differentiates the smoothed objective (LRH_NESTEROV)");
    if (p->max_k > 7) return fail(LRH_EUNSUPPORTED, "the adjoint kernels handle regions of at most 7 sites");
    DeviceGuard dg(p->device);
    const int64_t NI = p->n_inst;
    DevProblem& P = p->P;
    if (!P.thb) {
        int rc;
        if ((rc = p->dalloc(&P.thb, NI * p->all_elems)) || (rc = p->dalloc(&P.gbar, NI * p->msg_elems)) ||
            (rc = p->dalloc(&P.qbar, NI)) || (rc = p->dalloc(&p->vjp_nubar, NI * p->msg_elems)) ||
            (rc = p->dalloc(&p->vjp_termbar, NI * p->term_total)))
            return rc;
        std::vector<TermInfo> ti(std::max(p->n_terms, 1));
        for (int t = 0; t < p->n_terms; ++t) {
            ti[t].out_off = p->term_off[t];
            ti[t].region = p->term_region[t];
            ti[t].mask = p->term_mask[t];
            ti[t].kt = p->term_kt[t];
            ti[t].dr = 1 << p->region_k[p->term_region[t]];
        }
        TermInfo* dti;
        if ((rc = p->dalloc(&dti, (int64_t)ti.size()))) return rc;
        LRH_CK(cudaMemcpy(dti, ti.data(), sizeof(TermInfo) * ti.size(), cudaMemcpyHostToDevice));
        P.terms = dti;
        drop_graphs(p);   // captured graphs hold a copy of P without the adjoint buffers
    }
    LRH_CK(cudaMemcpyAsync(P.qbar, q_bar, sizeof(double) * NI, cudaMemcpyHostToDevice, p->stream));
    const size_t mbytes = sizeof(float2) * NI * p->msg_elems;
    if (mbytes) {
        if (g_bar) LRH_CK(cudaMemcpyAsync(P.gbar, g_bar, mbytes, g_bar_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, p->stream));
        else LRH_CK(cudaMemsetAsync(P.gbar, 0, mbytes, p->stream));
    }
    for (size_t c = 0; c < p->class_k.size(); ++c) {
        const int k = p->class_k[c];
        if (k >= 6) {
            if (!p->vjp_scratch) {   // scratch slots of the CTA adjoint: 2 D^2 complex per CTA of the launch
                int slots = 0;
                LRH_CK(vjp_cta_slots(p->max_k >= 7 ? 7 : 6, &slots));
                const int64_t D = (int64_t)1 << std::min(p->max_k, 7);
                int rc;
                if ((rc = p->dalloc(&p->vjp_scratch, (int64_t)slots * 2 * D * D))) return rc;
                p->vjp_slots = slots;
            }
            int slots = 0;
            LRH_CK(vjp_cta_slots(k, &slots));
            LRH_CK(launch_vjp_cta(P, k, p->class_list[c], p->class_count[c], p->vjp_scratch, std::min(slots, p->vjp_slots),
                                  p->stream));
        } else {
            LRH_CK(launch_vjp_region(P, k, p->class_list[c], p->class_count[c], p->stream));
        }
    }
    LRH_CK(launch_vjp_outputs(P, p->vjp_nubar, p->vjp_termbar, p->stream));
    const cudaMemcpyKind kind = out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (nu_bar && mbytes) LRH_CK(cudaMemcpyAsync(nu_bar, p->vjp_nubar, mbytes, kind, p->stream));
    if (term_bar && p->term_total)
        LRH_CK(cudaMemcpyAsync(term_bar, p->vjp_termbar, sizeof(float2) * NI * p->term_total, kind, p->stream));
    return read_err(p);
}

namespace {
struct StateHeader {
    uint64_t magic;        // "LRHSTAT1"
    int32_t n_inst;
    int32_t variant;
    int64_t msg_elems;
    int64_t iteration;
    int64_t warm_elems;
    lrh::IterState st;
};
constexpr uint64_t kStateMagic = 0x3154415453485231ull;
}  // namespace

int64_t lrh_state_bytes(const lrh_problem* p) {
    if (!p) return 0;
    return (int64_t)sizeof(StateHeader) + 3 * (int64_t)sizeof(float2) * p->n_inst * p->msg_elems +
           (int64_t)sizeof(double) * p->n_inst + (int64_t)sizeof(float2) * p->warm_elems;
}

int lrh_get_state(lrh_problem* p, void* buf, int64_t bytes) {
    if (!p || !buf) return fail(LRH_EINVAL, "NULL argument");
    if (bytes != lrh_state_bytes(p)) return fail(LRH_EINVAL, "bytes must equal lrh_state_bytes()");
    DeviceGuard dg(p->device);
    StateHeader h{};
    h.magic = kStateMagic;
    h.n_inst = p->n_inst;
    h.variant = p->opt.variant;
    h.msg_elems = p->msg_elems;
    h.iteration = p->iteration;
    h.warm_elems = p->warm_elems;
    char* out = static_cast<char*>(buf);
    const size_t m = sizeof(float2) * p->n_inst * p->msg_elems;
    LRH_CK(cudaMemcpyAsync(&h.st, p->P.st, sizeof(IterState), cudaMemcpyDeviceToHost, p->stream));
    char* q = out + sizeof(StateHeader);
    if (m) {
        LRH_CK(cudaMemcpyAsync(q, p->P.nu, m, cudaMemcpyDeviceToHost, p->stream));
        LRH_CK(cudaMemcpyAsync(q + m, p->P.zeta, m, cudaMemcpyDeviceToHost, p->stream));
        LRH_CK(cudaMemcpyAsync(q + 2 * m, p->P.nu_best, m, cudaMemcpyDeviceToHost, p->stream));
    }
    LRH_CK(cudaMemcpyAsync(q + 3 * m, p->P.q_best, sizeof(double) * p->n_inst, cudaMemcpyDeviceToHost, p->stream));
    if (p->warm_elems)
        LRH_CK(cudaMemcpyAsync(q + 3 * m + sizeof(double) * p->n_inst, p->P.warm, sizeof(float2) * p->warm_elems,
                               cudaMemcpyDeviceToHost, p->stream));
    LRH_CK(cudaStreamSynchronize(p->stream));
    std::memcpy(out, &h, sizeof(h));
    return LRH_OK;
}

int lrh_set_state(lrh_problem* p, const void* buf, int64_t bytes) {
    if (!p || !buf) return fail(LRH_EINVAL, "NULL argument");
    if (bytes != lrh_state_bytes(p)) return fail(LRH_EINVAL, "bytes must equal lrh_state_bytes()");
    StateHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (h.magic != kStateMagic || h.n_inst != p->n_inst || h.msg_elems != p->msg_elems || h.variant != p->opt.variant ||
        h.warm_elems != p->warm_elems)
        return fail(LRH_EINVAL, "state does not belong to a problem of this shape and variant");
    DeviceGuard dg(p->device);
    const char* q = static_cast<const char*>(buf) + sizeof(StateHeader);
    const size_t m = sizeof(float2) * p->n_inst * p->msg_elems;
    LRH_CK(cudaMemcpyAsync(p->P.st, &h.st, sizeof(IterState), cudaMemcpyHostToDevice, p->stream));
    if (m) {
        LRH_CK(cudaMemcpyAsync(p->P.nu, q, m, cudaMemcpyHostToDevice, p->stream));
        LRH_CK(cudaMemcpyAsync(p->P.zeta, q + m, m, cudaMemcpyHostToDevice, p->stream));
        LRH_CK(cudaMemcpyAsync(p->P.nu_best, q + 2 * m, m, cudaMemcpyHostToDevice, p->stream));
    }
    LRH_CK(cudaMemcpyAsync(p->P.q_best, q + 3 * m, sizeof(double) * p->n_inst, cudaMemcpyHostToDevice, p->stream));
    if (p->warm_elems)
        LRH_CK(cudaMemcpyAsync(p->P.warm, q + 3 * m + sizeof(double) * p->n_inst, sizeof(float2) * p->warm_elems,
                               cudaMemcpyHostToDevice, p->stream));
    LRH_CK(cudaStreamSynchronize(p->stream));
    p->iteration = h.iteration;
    return LRH_OK;
}

}  // extern "C"

namespace {

// Cache format: one JSON object per line, {"key": "...", "block": B} or {"key": "...", "concurrent": 0|1}.
std::vector<std::pair<std::string, int>> read_cache(const char* path) {
    std::vector<std::pair<std::string, int>> out;
    if (!path) return out;
    FILE* f = std::fopen(path, "r");
    if (!f) return out;
    char line[512];
    while (std::fgets(line, sizeof(line), f)) {
        std::string l(line);
        const size_t k0 = l.find("\"key\": \"");
        if (k0 == std::string::npos) continue;
        const size_t ks = k0 + 8, ke = l.find('"', ks);      // 8 = strlen("\"key\": \"")
        if (ke == std::string::npos) continue;
        const size_t c = l.find(':', ke + 1);               // the value after "block" / "concurrent"
        if (c == std::string::npos) continue;
        out.emplace_back(l.substr(ks, ke - ks), std::atoi(l.c_str() + c + 1));
    }
    std::fclose(f);
    return out;
}

int cache_lookup(const std::vector<std::pair<std::string, int>>& c, const std::string& key, int* val) {
    for (auto it = c.rbegin(); it != c.rend(); ++it)
        if (it->first == key) { *val = it->second; return 1; }
    return 0;
}

// Time `reps` calls of fn on the problem's stream with CUDA events (milliseconds per call).
template <typename F>
int time_ms(lrh_problem* p, int reps, F fn, float* ms) {
    struct Events {
        cudaEvent_t a = nullptr, b = nullptr;
        ~Events() { if (a) cudaEventDestroy(a); if (b) cudaEventDestroy(b); }
    } ev;
    LRH_CK(cudaEventCreate(&ev.a));
    LRH_CK(cudaEventCreate(&ev.b));
    int rc = fn();   // warm-up (and graph capture)
    if (rc) return rc;
    LRH_CK(cudaEventRecord(ev.a, p->stream));
    for (int i = 0; i < reps && !rc; ++i) rc = fn();
    if (rc) return rc;
    LRH_CK(cudaEventRecord(ev.b, p->stream));
    LRH_CK(cudaEventSynchronize(ev.b));
    float t = 0;
    LRH_CK(cudaEventElapsedTime(&t, ev.a, ev.b));
    *ms = t / reps;
    return LRH_OK;
}

// time_ms with enough repetitions for about `min_ms` of timed work (at least 2, at most 200):
// one call estimates the cost, so that microsecond-scale candidates are not compared on noise.
template <typename F>
int time_adaptive(lrh_problem* p, float min_ms, F fn, float* ms) {
    float est = 0.f;
    int rc = time_ms(p, 1, fn, &est);
    if (rc) return rc;
    int reps = est > 0.f ? (int)std::ceil(min_ms / est) : 200;
    reps = std::max(2, std::min(200, reps));
    return time_ms(p, reps, fn, ms);
}

}  // namespace

extern "C" {

namespace {
int autotune_impl(lrh_problem* p, const char* cache_path, int32_t flags);
}

int lrh_autotune(lrh_problem* p, const char* cache_path, int32_t flags) {
    if (!p) return fail(LRH_EINVAL, "NULL problem");
    if (p->has_ghost) return fail(LRH_EUNSUPPORTED, "problems with ghost regions iterate with lrh_halo_pass / lrh_halo_update");
    DeviceGuard dg(p->device);
    // the timing passes rewrite the stored eigenbases: keep a copy and put it back, so that a
    // run gives the same results whether or not it was tuned
    float2* keep = nullptr;
    const size_t wb = sizeof(float2) * (size_t)p->warm_elems;
    if (wb) {
        if (cudaMalloc(&keep, wb) != cudaSuccess) return fail(LRH_ENOMEM, "cudaMalloc (copy of the stored eigenbases)");
        if (cudaMemcpyAsync(keep, p->P.warm, wb, cudaMemcpyDeviceToDevice, p->stream) != cudaSuccess) {
            cudaFree(keep);
            return fail(LRH_ECUDA, "copy of the stored eigenbases");
        }
    }
    int rc = autotune_impl(p, cache_path, flags);
    if (keep) {
        const cudaError_t e1 = cudaMemcpyAsync(p->P.warm, keep, wb, cudaMemcpyDeviceToDevice, p->stream);
        const cudaError_t e2 = cudaStreamSynchronize(p->stream);
        cudaFree(keep);
        if (!rc && (e1 != cudaSuccess || e2 != cudaSuccess)) rc = fail(LRH_ECUDA, "restoring the stored eigenbases");
    }
    return rc;
}

namespace {
int autotune_impl(lrh_problem* p, const char* cache_path, int32_t flags) {
    int sms = 0;
    LRH_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
    const bool force = (flags & 1) != 0;
    if (!cache_path && p->opt.tune_cache) cache_path = p->opt.tune_cache;
    auto cache = force ? std::vector<std::pair<std::string, int>>() : read_cache(cache_path);
    std::vector<std::string> new_lines;
    for (size_t c = 0; c < p->class_k.size(); ++c) {
        const int k = p->class_k[c];
        if (k > 5) {   // CTA classes: one region per CTA; choose the back-transform (CUDA cores or tcgen05)
            const std::string key = "region_pass_backtransform k=" + std::to_string(k) + " units=" +
                                    std::to_string((int64_t)p->class_count[c] * p->n_inst) + " sms=" + std::to_string(sms);
            int mode = 0;
            if (!cache_lookup(cache, key, &mode)) {
                float best = 1e30f;
                for (int cand : {LRH_SHAPE_CTA_FP32, LRH_SHAPE_CTA_TENSOR}) {
                    if (cand == LRH_SHAPE_CTA_TENSOR && k != 7) continue;   // built for 7-site regions only
                    int rc = lrh_set_launch_shape(p, k, cand);
                    if (rc) return rc;
                    float ms = 0;
                    rc = time_adaptive(p, 2.0f, [&]() -> int {
                        LRH_CK(launch_region_pass(p->P, plain_io(p), k, p->class_list[c], p->class_count[c], p->stream, 0));
                        return LRH_OK; }, &ms);
                    if (rc) return rc;
                    if (ms < best) { best = ms; mode = cand; }
                }
                new_lines.push_back("{\"key\": \"" + key + "\", \"block\": " + std::to_string(mode) + "}");
            }
            int rc = lrh_set_launch_shape(p, k, mode);
            if (rc) return rc;
            continue;
        }
        // with stored eigenbases the 3- and 4-site classes are tuned among the 2x2-block shapes
        // only, the layout that warm-starts: passes timed at one point cannot see the sweeps the
        // warm starts save from one iteration to the next (at nu = 0 every layout is trivial)
        const bool warm_k = (k == 3 || k == 4) && p->P.warm != nullptr && p->P.warm_off[k] >= 0 && !p->opt.cold_start;
        const std::string key = "region_pass k=" + std::to_string(k) + " units=" +
                                std::to_string((int64_t)p->class_count[c] * p->n_inst) + " sms=" + std::to_string(sms) +
                                (warm_k ? " warm" : "");
        int blk = 0;
        if (!cache_lookup(cache, key, &blk)) {
            float best = 1e30f;
            for (int cand : {64, 128, 256, -64, -128, -256, LRH_SHAPE_BLOCKS + 64, LRH_SHAPE_BLOCKS + 128,
                             LRH_SHAPE_BLOCKS + 256, LRH_SHAPE_WARP16 + 64, LRH_SHAPE_WARP16 + 128, LRH_SHAPE_WARP16 + 256}) {
                if (cand > 0 && cand < LRH_SHAPE_BLOCKS && cand < (1 << k)) continue;
                if (cand < 0 && k != 2) continue;   // thread-per-region layout: 4 x 4 regions
                if (cand > LRH_SHAPE_BLOCKS && cand < LRH_SHAPE_WARP16 && k != 3 && k != 4) continue;   // 8 x 8, 16 x 16
                if (cand > LRH_SHAPE_WARP16 && k != 4) continue;   // one warp per 16 x 16 region
                if (warm_k && !(cand > LRH_SHAPE_BLOCKS && cand < LRH_SHAPE_WARP16)) continue;
                float ms = 0;
                int rc = time_adaptive(p, 2.0f, [&]() -> int {
                    LRH_CK(launch_region_pass(p->P, plain_io(p), k, p->class_list[c], p->class_count[c], p->stream, cand));
                    return LRH_OK; }, &ms);
                if (rc) return rc;
                if (ms < best) { best = ms; blk = cand; }
            }
            new_lines.push_back("{\"key\": \"" + key + "\", \"block\": " + std::to_string(blk) + "}");
        }
        p->class_block[c] = blk;
    }
    layout_plan(p);
    // Iteration driver: how the classes of a pass are launched (one after another, forked
    // streams, one launch) under the graph driver, and the persistent driver; each timed over
    // whole iterations on a saved copy of the multipliers and iteration scalars.
    const bool several = p->class_k.size() > 1;
    if (several || p->persist_grid > 0) {
        drop_graphs(p);
        std::string key = std::string("driver variant=") + (p->opt.variant == LRH_NESTEROV ? "nesterov" : "subgradient");
        for (size_t c = 0; c < p->class_k.size(); ++c)
            key += " k" + std::to_string(p->class_k[c]) + "=" + std::to_string((int64_t)p->class_count[c] * p->n_inst) +
                   "/" + std::to_string(p->class_block[c]);
        key += " sms=" + std::to_string(sms);
        int choice = 10 * LRH_LOOP_GRAPH + 1;   // 10 * loop + class mode
        if (!cache_lookup(cache, key, &choice)) {
            const int64_t nm = p->n_inst * p->msg_elems;
            const size_t b_msg = sizeof(float2) * (size_t)std::max<int64_t>(nm, 1);
            const size_t b_inst = sizeof(double) * (size_t)p->n_inst;
            struct Scratch {
                void* ptr = nullptr;
                ~Scratch() { if (ptr) cudaFree(ptr); }
            } scratch;
            LRH_CK(cudaStreamSynchronize(p->stream));
            if (cudaMalloc(&scratch.ptr, 3 * b_msg + 2 * b_inst + sizeof(IterState) + 64) != cudaSuccess)
                return fail(LRH_ENOMEM, "cudaMalloc of the autotuner's saved multipliers failed");
            char* base = static_cast<char*>(scratch.ptr);
            float2* s_nu = reinterpret_cast<float2*>(base);
            float2* s_zeta = reinterpret_cast<float2*>(base + b_msg);
            float2* s_best = reinterpret_cast<float2*>(base + 2 * b_msg);
            double* s_q = reinterpret_cast<double*>(base + 3 * b_msg);
            int32_t* s_flag = reinterpret_cast<int32_t*>(base + 3 * b_msg + b_inst);
            IterState* s_st = reinterpret_cast<IterState*>(base + 3 * b_msg + 2 * b_inst);
            auto copy_all = [&](bool save) -> int {
                auto cp = [&](void* x, void* y, size_t bytes) {
                    return cudaMemcpyAsync(save ? x : y, save ? y : x, bytes, cudaMemcpyDeviceToDevice, p->stream);
                };
                LRH_CK(cp(s_nu, p->P.nu, sizeof(float2) * nm));
                LRH_CK(cp(s_zeta, p->P.zeta, sizeof(float2) * nm));
                LRH_CK(cp(s_best, p->P.nu_best, sizeof(float2) * nm));
                LRH_CK(cp(s_q, p->P.q_best, sizeof(double) * p->n_inst));
                LRH_CK(cp(s_flag, p->P.best_flag, sizeof(int32_t) * p->n_inst));
                LRH_CK(cp(s_st, p->P.st, sizeof(IterState)));
                return LRH_OK;
            };
            const int saved_loop = p->opt.loop;
            const bool saved_conc = p->concurrent, saved_fused = p->fused;
            const int64_t saved_it = p->iteration;
            constexpr int kTuneIters = 8;
            int rc;
            if ((rc = copy_all(true))) return rc;
            float best = 1e30f;
            for (int cand = 0; cand < 4; ++cand) {   // graph x {0, 1, 2}, then persistent
                const int loop = cand < 3 ? LRH_LOOP_GRAPH : LRH_LOOP_PERSISTENT;
                const int mode = cand < 3 ? cand : 1;
                if (cand < 3 && !several && mode != 1) continue;
                if (cand == 2 && p->persist_grid <= 0) continue;
                if (cand == 3 && p->persist_grid <= 0) continue;
                p->opt.loop = loop;
                p->concurrent = mode == 1;
                p->fused = mode == 2;
                drop_graphs(p);
                float ms = 0;
                rc = time_adaptive(p, 4.0f, [&]() { return lrh_step(p, kTuneIters); }, &ms);
                const int rc2 = copy_all(false);
                p->iteration = saved_it;
                if (rc || rc2) {
                    p->opt.loop = saved_loop; p->concurrent = saved_conc; p->fused = saved_fused;
                    return rc ? rc : rc2;
                }
                if (ms < best) { best = ms; choice = 10 * loop + mode; }
            }
            p->opt.loop = saved_loop;
            LRH_CK(cudaStreamSynchronize(p->stream));
            new_lines.push_back("{\"key\": \"" + key + "\", \"driver\": " + std::to_string(choice) + "}");
        }
        const int loop = choice / 10, mode = choice % 10;
        p->concurrent = mode == 1;
        p->fused = mode == 2 && p->persist_grid > 0;
        p->loop_auto = (loop == LRH_LOOP_PERSISTENT && p->persist_grid > 0) ? LRH_LOOP_PERSISTENT : LRH_LOOP_GRAPH;
        drop_graphs(p);
    }
    if (cache_path && !new_lines.empty()) {
        FILE* f = std::fopen(cache_path, "a");
        if (!f) return fail(LRH_EINVAL, std::string("cannot write the autotune cache ") + cache_path);
        for (auto& l : new_lines) std::fprintf(f, "%s\n", l.c_str());
        std::fclose(f);
    }
    drop_graphs(p);   // captured launch shapes are stale
    return read_err(p);
}
}  // namespace

int lrh_set_launch_shape(lrh_problem* p, int32_t k_sites, int32_t block) {
    if (!p) return fail(LRH_EINVAL, "NULL problem");
    bool ok;
    if (k_sites >= 6) ok = block == LRH_SHAPE_CTA_FP32 || (block == LRH_SHAPE_CTA_TENSOR && k_sites == 7);
    else if (block > LRH_SHAPE_WARP16)
        ok = k_sites == 4 && (block - LRH_SHAPE_WARP16 == 64 || block - LRH_SHAPE_WARP16 == 128 ||
                              block - LRH_SHAPE_WARP16 == 256);
    else if (block > LRH_SHAPE_BLOCKS)
        ok = (k_sites == 3 || k_sites == 4) && (block - LRH_SHAPE_BLOCKS == 64 || block - LRH_SHAPE_BLOCKS == 128 ||
                                                block - LRH_SHAPE_BLOCKS == 256);
    else ok = (block == 64 || block == 128 || block == 256 || (k_sites == 2 && (block == -64 || block == -128 || block == -256))) &&
              !(block > 0 && block < (1 << k_sites));
    if (!ok) return fail(LRH_EINVAL, "unsupported launch shape for this region size");
    for (size_t c = 0; c < p->class_k.size(); ++c)
        if (p->class_k[c] == k_sites) {
            p->class_block[c] = block;
            if (k_sites >= 6) {
                const int bit = 1 << (k_sites - 6);
                p->P.tc_backtransform = block == LRH_SHAPE_CTA_TENSOR ? (p->P.tc_backtransform | bit) : (p->P.tc_backtransform & ~bit);
            }
            layout_plan(p);
            drop_graphs(p);
            return LRH_OK;
        }
    return fail(LRH_EINVAL, "no region class with " + std::to_string(k_sites) + " sites");
}

int lrh_set_class_mode(lrh_problem* p, int32_t mode) {
    if (!p) return fail(LRH_EINVAL, "NULL problem");
    if (mode < 0 || mode > 2) return fail(LRH_EINVAL, "class mode must be 0, 1 or 2");
    if (mode == 2 && p->persist_grid <= 0) return fail(LRH_EUNSUPPORTED, "one-launch passes need classes of <= 4 sites");
    p->concurrent = mode == 1;
    p->fused = mode == 2;
    drop_graphs(p);
    return LRH_OK;
}

int lrh_selftest_barrier_timeout(lrh_problem* p) {
    if (!p) return fail(LRH_EINVAL, "NULL problem");
    if (p->persist_grid <= 0) return fail(LRH_EUNSUPPORTED, "this problem has no persistent launch");
    DeviceGuard dg(p->device);
    int rc = read_err(p);
    if (rc) return rc;
    PersistPlan L = p->plan;
    L.n = 1;
    L.nesterov = p->opt.variant == LRH_NESTEROV ? 1 : 0;
    L.par0 = (int)(p->iteration & 1);
    LRH_CK(launch_persistent(p->P, L, p->persist_kmax, p->persist_grid, p->stream, true));
    return read_err(p);
}

int lrh_synchronize(lrh_problem* p) {
    if (!p) return fail(LRH_EINVAL, "NULL problem");
    DeviceGuard dg(p->device);
    return read_err(p);
}

}  // extern "C"

extern "C" {

int lrh_theorem_parameters(const lrh_problem* p, double eps, double R, double c_frac, lrh_params* out) {
    if (!p || !out) return fail(LRH_EINVAL, "NULL argument");
    if (!(eps > 0.0) || !std::isfinite(eps)) return fail(LRH_EINVAL, "eps must be finite and > 0");
    if (!(c_frac > 0.0 && c_frac < 1.0)) return fail(LRH_EINVAL, "c_frac must lie in (0, 1)");
    const double n = (double)p->n_sites;
    lrh_params r{};
    r.n_sites = p->n_sites;
    r.lambda_G = p->lambda_G;
    r.gamma_G = p->gamma_G;
    r.kappa_G = p->kappa;
    r.beta = 2.0 * p->gamma_G / (n * eps);                     // Thm 5 / Thm 7: smoothing error eps/2
    r.lhat = r.beta * p->lambda_G / 2.0;
    r.c = c_frac / std::max(1, p->kappa);                      // Thm 4 / Thm 6: 0 < c < 1 / kappa_G
    r.alpha = r.c * eps;
    r.T_nesterov = -1;
    r.T_subgradient = -1;
    if (R > 0.0 && std::isfinite(R)) {
        r.T_nesterov = (int64_t)std::ceil(2.0 * R * std::sqrt(p->gamma_G * p->lambda_G) / (n * eps)) - 1;
        r.T_subgradient = (int64_t)std::ceil(R * R / (2.0 * r.c * (1.0 - r.c * p->kappa) * n * eps * eps));
    }
    *out = r;
    return LRH_OK;
}

int lrh_reset(lrh_problem* p) {
    if (!p) return fail(LRH_EINVAL, "NULL problem");
    DeviceGuard dg(p->device);
    const size_t m = sizeof(float2) * (size_t)p->n_inst * (size_t)p->msg_elems;
    if (m) {
        LRH_CK(cudaMemsetAsync(p->P.nu, 0, m, p->stream));
        LRH_CK(cudaMemsetAsync(p->P.zeta, 0, m, p->stream));
        LRH_CK(cudaMemsetAsync(p->P.nu_best, 0, m, p->stream));
    }
    std::vector<double> ninf(p->n_inst, -std::numeric_limits<double>::infinity());
    LRH_CK(cudaMemcpyAsync(p->P.q_best, ninf.data(), sizeof(double) * p->n_inst, cudaMemcpyHostToDevice, p->stream));
    LRH_CK(cudaMemsetAsync(p->P.best_flag, 0, sizeof(int32_t) * p->n_inst, p->stream));
    int rc = push_state(p, true, 1.0, 0.0);
    if (rc) return rc;
    if ((rc = reset_warm(p))) return rc;
    LRH_CK(cudaStreamSynchronize(p->stream));   // the host vector above must outlive the copy
    return LRH_OK;
}

namespace {
// FP32 estimate of Q(nu) = sum_e lambda_min(theta_e(nu)) per instance: one region pass in the
// ground-state mode at nu (no update; the pass's states and traces are rewritten by the next
// iteration's first pass), FP64 sums.  Restores the iteration scalars' mode afterwards.
int estimate_q32(lrh_problem* p, double* out) {
    const lrh_options& o = p->opt;
    const double degen = o.degen_tol > 0.0 ? o.degen_tol : 1e-5;
    const int sweeps = o.max_sweeps > 0 ? o.max_sweeps : 15;
    const int cert = o.cert_sweeps > 0 ? o.cert_sweeps : 40;
    LRH_CK(launch_set_state(p->P, (int)(p->iteration & 1), 0.0, 0.0, 0, o.beta, 1.0 / p->lhat_eff, o.alpha, degen,
                            LRH_SUBGRADIENT, o.step_rule, sweeps, cert, 1, p->stream));   // cold: stored bases untouched
    PassIO io{};
    io.nu_in = p->P.nu;
    io.rho_out = p->P.rho;
    io.tr_out = p->P.tr;
    int rc = launch_all_classes(p, io);
    if (rc) return rc;
    LRH_CK(launch_reduce(p->P, p->P.val, 0, p->stream));
    LRH_CK(cudaMemcpyAsync(p->h_pinned, p->P.q_sum, sizeof(double) * p->n_inst, cudaMemcpyDeviceToHost, p->stream));
    if ((rc = push_state(p, false, 0.0, 0.0))) return rc;
    if ((rc = read_err(p))) return rc;
    std::copy(p->h_pinned, p->h_pinned + p->n_inst, out);
    return LRH_OK;
}
}  // namespace

int lrh_solve(lrh_problem* p, int32_t max_records, lrh_record* rec, double* rec_bounds, int32_t* n_records,
              double* bound_out) {
    if (!p || !bound_out) return fail(LRH_EINVAL, "NULL argument");
    if (p->has_ghost) return fail(LRH_EUNSUPPORTED, "problems with ghost regions iterate with lrh_halo_pass / lrh_halo_update");
    if (max_records < 0 || (max_records > 0 && (!rec || !rec_bounds))) return fail(LRH_EINVAL, "bad record buffers");
    DeviceGuard dg(p->device);
    const auto t0 = std::chrono::steady_clock::now();
    const int64_t NI = p->n_inst;
    std::vector<double> cur((size_t)NI);
    int32_t nrec = 0;
    int64_t done = 0;
    int status = LRH_OK;
    bool stop = false, reached = false;
    if (n_records) *n_records = 0;
    const bool targeted = !p->target.empty() && p->opt.certify_every > 0;
    std::vector<double> est((size_t)NI);
    auto record = [&](double beta, bool last) -> int {
        if (targeted && p->opt.screen_tol > 0.0 && !last) {   // FP32 screen before the FP64 certificate
            int r = estimate_q32(p, est.data());
            if (r) return r;
            for (int64_t i = 0; i < NI; ++i)
                if (std::isfinite(p->target[i]) && est[i] < p->target[i] - p->opt.screen_tol) return LRH_OK;
        }
        int r = lrh_bound(p, LRH_BOUND_CERTIFIED, cur.data());
        if (r && r != LRH_ENOCONV) return r;
        if (r == LRH_ENOCONV) status = LRH_ENOCONV;
        const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (nrec < max_records) {
            rec[nrec] = lrh_record{done, secs, beta};
            std::copy(cur.begin(), cur.end(), rec_bounds + (int64_t)nrec * NI);
            ++nrec;
            if (n_records) *n_records = nrec;
        }
        std::copy(cur.begin(), cur.end(), bound_out);
        if (p->opt.deadline_s > 0.0 && secs > p->opt.deadline_s) stop = true;
        if (targeted) {
            bool all = true;
            for (int64_t i = 0; i < NI; ++i)
                if (std::isfinite(p->target[i]) && !(cur[i] >= p->target[i])) all = false;
            if (all) reached = true;
        }
        return LRH_OK;
    };
    const int per = p->opt.iters_per_stage;
    const int every = p->opt.certify_every > 0 ? p->opt.certify_every : std::max(per, 1);
    int rc;
    if (p->opt.variant == LRH_NESTEROV) {
        std::vector<double> stages = p->beta_sched;
        if (stages.empty()) stages.push_back(p->opt.beta);
        for (size_t si = 0; si < stages.size() && !stop && !reached; ++si) {
            p->opt.beta = stages[si];        // L_hat follows: lhat if set, else beta Lambda_G / 2
            if ((rc = lrh_restart(p))) return rc;
            for (int it = 0; it < per && !stop && !reached;) {
                const int n = std::min(every, per - it);
                if ((rc = lrh_step(p, n))) return rc;
                it += n;
                done += n;
                const bool last = si + 1 == stages.size() && it >= per;
                if (p->opt.certify_every > 0 && (rc = record(stages[si], last))) return rc;
            }
        }
        if (p->opt.certify_every <= 0 && (rc = record(p->opt.beta, true))) return rc;
    } else {
        if ((rc = lrh_restart(p))) return rc;
        for (int it = 0; it < per && !stop && !reached;) {
            const int n = std::min(every, per - it);
            if ((rc = lrh_step(p, n))) return rc;
            it += n;
            done += n;
            if (p->opt.certify_every > 0 && (rc = record(0.0, it >= per))) return rc;
        }
        if (p->opt.certify_every <= 0 && (rc = record(0.0, true))) return rc;
    }
    if (stop) return fail(LRH_EDEADLINE, "lrh_solve reached its deadline");
    return status;
}

int lrh_plan_poset(const lrh_problem_desc* desc, int64_t pair_cap, int32_t* pair_parent, int32_t* pair_child,
                   int64_t* n_pairs, int32_t* term_region, double* lambda_G) {
    if (!desc) return fail(LRH_EINVAL, "desc is NULL");
    PosetPlan pl;
    int rc = plan_poset(desc, pl);
    if (rc) return rc;
    if (n_pairs) *n_pairs = pl.n_pairs;
    if (lambda_G) *lambda_G = pl.lambda_G;
    if (term_region) std::copy(pl.place.begin(), pl.place.end(), term_region);
    if (pair_parent || pair_child) {
        if (pair_cap < pl.n_pairs) return fail(LRH_EINVAL, "pair_cap is below the number of pairs");
        int64_t q = 0;
        for (int e = 0; e < desc->n_regions; ++e)
            for (auto& f : pl.kids[e]) {
                if (pair_parent) pair_parent[q] = e;
                if (pair_child) pair_child[q] = f.first;
                ++q;
            }
    }
    return LRH_OK;
}

int lrh_halo_set(lrh_problem* p, int32_t n_send, const lrh_halo_item* send, int32_t n_recv, const lrh_halo_item* recv,
                 int64_t* send_elems, int64_t* recv_elems) {
    if (!p || n_send < 0 || n_recv < 0 || (n_send > 0 && !send) || (n_recv > 0 && !recv))
        return fail(LRH_EINVAL, "bad arguments to lrh_halo_set");
    if (!p->has_ghost) return fail(LRH_EINVAL, "lrh_halo_set: the problem has no ghost regions");
    DeviceGuard dg(p->device);
    // rho offset of every region with a parent (-1 otherwise), from the pair table
    std::vector<int64_t> rho_off(p->n_regions, -1);
    {
        std::vector<RegionInfo> ri(p->n_regions);
        LRH_CK(cudaMemcpy(ri.data(), p->P.reg, sizeof(RegionInfo) * ri.size(), cudaMemcpyDeviceToHost));
        for (int e = 0; e < p->n_regions; ++e) rho_off[e] = ri[e].rho_off;
    }
    auto build = [&](const lrh_halo_item* it, int32_t n, bool incoming, std::vector<int64_t>& map) -> int {
        map.clear();
        for (int32_t i = 0; i < n; ++i) {
            const int32_t id = it[i].id;
            int64_t off, elems;
            if (it[i].kind == LRH_HALO_STATE) {
                if (id < 0 || id >= p->n_regions) return fail(LRH_EINVAL, "halo state item: region out of range");
                if (rho_off[id] < 0) return fail(LRH_EINVAL, "halo state item: region " + std::to_string(id) + " is no pair's child");
                if ((p->ghost[id] != 0) != incoming)
                    return fail(LRH_EINVAL, std::string("halo state item: region ") + std::to_string(id) +
                                                (incoming ? " is not a ghost (only ghost states are received)"
                                                          : " is a ghost (only owned states are sent)"));
                off = rho_off[id];
                elems = (int64_t)1 << (2 * p->region_k[id]);
            } else if (it[i].kind == LRH_HALO_TRACE) {
                if (id < 0 || id >= p->n_pairs) return fail(LRH_EINVAL, "halo trace item: pair out of range");
                const int par = p->pair_parent[id];
                if ((p->ghost[par] != 0) != incoming)
                    return fail(LRH_EINVAL, std::string("halo trace item: pair ") + std::to_string(id) +
                                                (incoming ? " has an owned parent (only traces of ghost parents are received)"
                                                          : " has a ghost parent (only traces of owned parents are sent)"));
                off = ~p->pair_off[id];
                elems = (int64_t)1 << (2 * p->region_k[p->pair_child[id]]);
            } else {
                return fail(LRH_EINVAL, "halo item of unknown kind");
            }
            for (int64_t c = 0; c < elems / 4; ++c) map.push_back(off >= 0 ? off + 4 * c : ~(~off + 4 * c));
        }
        return LRH_OK;
    };
    std::vector<int64_t> smap, rmap;
    int rc;
    if ((rc = build(send, n_send, false, smap)) || (rc = build(recv, n_recv, true, rmap))) return rc;
    // every ghost state and every ghost-parent trace the update reads is received exactly once
    {
        std::vector<int32_t> got_state(p->n_regions, 0), got_trace(p->n_pairs, 0);
        for (int32_t i = 0; i < n_recv; ++i) (recv[i].kind == LRH_HALO_STATE ? got_state[recv[i].id] : got_trace[recv[i].id])++;
        for (int e = 0; e < p->n_regions; ++e)
            if (p->ghost[e] && rho_off[e] >= 0 && got_state[e] != 1)
                return fail(LRH_EINVAL, "ghost region " + std::to_string(e) + " state is received " + std::to_string(got_state[e]) +
                                            " times (exactly once needed)");
        for (int q = 0; q < p->n_pairs; ++q)
            if (p->ghost[p->pair_parent[q]] && got_trace[q] != 1)
                return fail(LRH_EINVAL, "pair " + std::to_string(q) + " (ghost parent) trace is received " +
                                            std::to_string(got_trace[q]) + " times (exactly once needed)");
    }
    p->dfree(p->halo_send);
    p->dfree(p->halo_recv);
    p->halo_send = p->halo_recv = nullptr;
    p->halo_ready = false;
    if ((rc = p->dalloc(&p->halo_send, (int64_t)smap.size())) || (rc = p->dalloc(&p->halo_recv, (int64_t)rmap.size()))) return rc;
    if (!smap.empty()) LRH_CK(cudaMemcpy(p->halo_send, smap.data(), sizeof(int64_t) * smap.size(), cudaMemcpyHostToDevice));
    if (!rmap.empty()) LRH_CK(cudaMemcpy(p->halo_recv, rmap.data(), sizeof(int64_t) * rmap.size(), cudaMemcpyHostToDevice));
    p->halo_send_chunks = (int64_t)smap.size();
    p->halo_recv_chunks = (int64_t)rmap.size();
    p->halo_ready = true;
    if (send_elems) *send_elems = 4 * p->halo_send_chunks;
    if (recv_elems) *recv_elems = 4 * p->halo_recv_chunks;
    return LRH_OK;
}

int lrh_halo_pass(lrh_problem* p) {
    if (!p) return fail(LRH_EINVAL, "NULL problem");
    if (p->opt.variant != LRH_NESTEROV) return fail(LRH_EUNSUPPORTED, "sharded iterations run Alg. 2 (LRH_NESTEROV) only");
    if (!p->halo_ready) return fail(LRH_EINVAL, "lrh_halo_set has not been called");
    DeviceGuard dg(p->device);
    // the first pass of lrh_step: canonical nu, zeta in; states and traces to the X arenas
    PassIO io{};
    io.rel = 0;
    io.writer = 1;
    io.pending = 0;
    io.nu_in = p->P.nu;
    io.zeta_in = p->P.zeta;
    io.rho_out = p->P.rho;
    io.tr_out = p->P.tr;
    int rc = launch_all_classes(p, io);
    if (rc) return rc;
    p->halo_passed = true;
    return LRH_OK;
}

int lrh_halo_pack(lrh_problem* p, void* send) {
    if (!p || (!send && p->halo_send_chunks > 0)) return fail(LRH_EINVAL, "NULL argument");
    if (!p->halo_ready) return fail(LRH_EINVAL, "lrh_halo_set has not been called");
    if ((reinterpret_cast<uintptr_t>(send) & 15) != 0) return fail(LRH_EINVAL, "halo buffer must be 16-byte aligned");
    DeviceGuard dg(p->device);
    if (p->halo_send_chunks) LRH_CK(launch_halo_copy(p->P, p->halo_send, p->halo_send_chunks, static_cast<float2*>(send), 0, p->stream));
    return LRH_OK;
}

int lrh_halo_unpack(lrh_problem* p, const void* recv) {
    if (!p || (!recv && p->halo_recv_chunks > 0)) return fail(LRH_EINVAL, "NULL argument");
    if (!p->halo_ready) return fail(LRH_EINVAL, "lrh_halo_set has not been called");
    if ((reinterpret_cast<uintptr_t>(recv) & 15) != 0) return fail(LRH_EINVAL, "halo buffer must be 16-byte aligned");
    DeviceGuard dg(p->device);
    if (p->halo_recv_chunks)
        LRH_CK(launch_halo_copy(p->P, p->halo_recv, p->halo_recv_chunks, const_cast<float2*>(static_cast<const float2*>(recv)), 1,
                                p->stream));
    return LRH_OK;
}

int lrh_halo_update(lrh_problem* p) {
    if (!p) return fail(LRH_EINVAL, "NULL problem");
    if (!p->halo_passed) return fail(LRH_EINVAL, "lrh_halo_update needs a preceding lrh_halo_pass");
    DeviceGuard dg(p->device);
    int rc = enqueue_nesterov_tail(p, 1);   // the Alg. 2 update of every message from the X arenas
    if (rc) return rc;
    p->halo_passed = false;
    p->iteration += 1;
    return LRH_OK;
}

}  // extern "C"
