// Internal device-side layout of an lrh problem (not part of the C ABI).
#pragma once
#include <cstdint>
#include <string>
#include <cuda_runtime.h>

namespace lrh {

// One region of the cluster family (identical for every batched instance).
struct RegionInfo {
    int64_t h_off;         // complex offset of D x D h_e in one instance's h arena, -1 = no term
    int64_t rho_off;       // complex offset of D x D rho_e in one instance's state arena, -1 = no parent
    int32_t child_begin;   // [child_begin, child_end) into child_pairs: pairs e->f with e = this
    int32_t child_end;
    int32_t parent_begin;  // [parent_begin, parent_end) into parent_pairs: pairs g->e with e = this
    int32_t parent_end;
    int64_t all_off;       // complex offset of D x D in an arena holding every region (adjoint)
};

// One Hamiltonian term, for the adjoint's term cotangents.
struct TermInfo {
    int64_t out_off;       // complex offset of the D_t x D_t block in one instance's term array
    int32_t region;        // region the term is placed in
    int32_t mask;          // bits of the region's basis index that carry the term's sites
    int32_t kt;            // term sites
    int32_t dr;            // D of the region holding the term
};

// One covering pair e -> f.
struct PairInfo {
    int64_t off;           // complex offset of the D_f x D_f message block in one instance
    int32_t parent;
    int32_t child;
    int32_t mask;          // bits of the parent's basis index that carry the child's sites
    int32_t kf;            // child sites
    int64_t child_rho;     // offset of the child's state rho_f in one instance's state arena
};

// Scalars of the iteration, double-buffered by iteration parity so that a captured
// graph of iterations needs no host-side argument changes.
struct IterState {
    double theta[2];       // Alg. 1 path: parity slots (unused by Alg. 2)
    double t[2];           // iterations since the last restart (Alg. 1 step-size rule)
    double th3[3];         // Alg. 2: theta_t in slot t mod 3 (a pass reads t-1 and t, writes t+1)
    long long t0;          // Alg. 2: iterations since the last restart, before the current lrh_step
    double beta;
    double inv_lhat;
    double alpha;
    double degen_tol;
    int32_t variant;
    int32_t step_rule;
    int32_t max_sweeps;
    int32_t cert_sweeps;   // sweep cap of the FP64 certification Jacobi
    int32_t cold;          // nonzero: eigensolves start from the identity (stored bases unused)
    int32_t pad_;
};

// Inputs and outputs of one region pass.  A "pending" pass first applies the previous
// iteration's Alg. 2 update to every message it gathers (g = rho_in_f - tr_in, zeta += g /
// (theta_{t-1} L_hat), nu = (1 - theta_{t-1}) nu + theta_{t-1} zeta); the region that is the
// child of a pair owns that message and writes the updated nu, zeta to nu_out / zeta_out.
struct PassIO {
    const float2* nu_in;
    const float2* zeta_in;   // nullptr: Alg. 1 (eta = nu)
    const float2* rho_in;
    const float2* tr_in;
    float2* nu_out;
    float2* zeta_out;
    float2* rho_out;
    float2* tr_out;
    int32_t rel;             // iteration t = st->t0 + rel
    int32_t pending;
    int32_t writer;          // this launch writes th3[(t + 1) mod 3]
    int32_t pad;
};

// Record of region i of a uniform class of size D (see DevProblem::class_first).
__host__ __device__ inline RegionInfo uniform_region(const RegionInfo& f, int64_t i, int64_t D2) {
    RegionInfo R = f;
    const int32_t nc = f.child_end - f.child_begin, np = f.parent_end - f.parent_begin;
    R.child_begin = f.child_begin + (int32_t)(i * nc);
    R.child_end = R.child_begin + nc;
    R.parent_begin = f.parent_begin + (int32_t)(i * np);
    R.parent_end = R.parent_begin + np;
    if (f.h_off >= 0) R.h_off = f.h_off + i * D2;
    if (f.rho_off >= 0) R.rho_off = f.rho_off + i * D2;
    R.all_off = f.all_off + i * D2;
    return R;
}

// Error bits raised by kernels.  DEV_ERR_NOCONV: an FP64 certification Jacobi stopped at its
// sweep cap with off-diagonal mass above the convergence threshold (its value is still a valid
// lower bound: the Weyl correction below covers the remaining off-diagonal part).
enum : int32_t { DEV_ERR_NUMERIC = 1, DEV_ERR_TIMEOUT = 2, DEV_ERR_NOCONV = 4 };

// Arrays indexed by a region's site count k (0 .. 8, regions of up to 8 sites).
constexpr int kClassSlots = 9;

struct DevProblem {
    int32_t n_inst;
    int32_t n_regions;
    int32_t n_pairs;
    int32_t tc_backtransform;   // bit k - 6 set: the D = 2^k CTA pass forms rho on the tensor cores
    int64_t h_elems;       // complex entries per instance
    int64_t rho_elems;
    int64_t msg_elems;
    const RegionInfo* reg;
    const PairInfo* pair;
    const int32_t* child_pairs;
    const int32_t* parent_pairs;
    const int32_t* chunk_pair;   // [msg_elems / 4] pair owning complex entries 4c .. 4c+3
    const int64_t* chunk_rho;    // [msg_elems / 4] child-state offset minus message offset of that pair
    const PairInfo* child_info;  // PairInfo in child CSR order (child_pairs[q] resolved)
    const PairInfo* parent_info; // PairInfo in parent CSR order
    int32_t class_base[kClassSlots];   // [k]: first region id when the class of k sites is a contiguous id range, else -1
    // [k]: record of the class's first region when every region r = class_base[k] + i of the class
    // has the record of the first shifted by i (child / parent ranges by their lengths, term and
    // state offsets by D^2 where present); lets the small-region passes build the record without
    // a dependent load.  class_uniform bit k marks such classes.
    RegionInfo class_first[kClassSlots];
    int32_t class_uniform;
    const float2* h32;     // [n_inst][h_elems]
    const double2* h64;    // [n_inst][h_elems]
    float2* nu;            // [n_inst][msg_elems]
    float2* zeta;
    float2* nu_best;
    float2* tr;            // Tr_{e\f} rho_e of the last pass, message layout
    float2* rho;           // [n_inst][rho_elems] states of regions that have parents
    float2* grad;          // gradient of the last lrh_evaluate
    float2* nu_b;          // second buffers of the fused Alg. 2 iteration (ping-pong)
    float2* zeta_b;
    float2* rho_b;
    float2* tr_b;
    double* val;           // [n_inst][n_regions] per-region FP32 values of the last pass
    double* val64;         // [n_inst][n_regions] per-region FP64 lambda_min of the last certify
    double* q_sum;         // [n_inst] scratch sums
    double* q_best;        // [n_inst]
    int32_t* best_flag;    // [n_inst]
    IterState* st;
    int32_t* err;
    unsigned long long* sweeps;   // [kClassSlots] per size class (indexed by k)
    unsigned long long* capped;   // [kClassSlots] per size class: FP32 eigensolves stopped by the sweep cap
    // adjoint (allocated on the first lrh_vjp call)
    int64_t all_elems;     // complex entries of the every-region arena per instance
    int32_t n_terms;
    int32_t pad2;
    int64_t term_total;    // complex entries of one instance's term array
    const TermInfo* terms;
    float2* thb;           // [n_inst][all_elems] theta_bar of every region
    float2* gbar;          // [n_inst][msg_elems] cotangent of the gradient output
    double* qbar;          // [n_inst] cotangent of Q_beta
    // regions of 8 sites (D = 256): one global scratch slot per CTA of their launch (theta
    // entries beyond shared memory, V, rho and the rotation log), allocated at creation
    float2* big;
    int64_t big_slot;        // complex entries per slot
    int32_t big_slots;       // slots (= CTAs of a D = 256 launch)
    int32_t big_log_sweeps;  // sweeps the rotation log of a slot holds (the D = 256 sweep cap)
    // stored eigenbases of the 2x2-block classes (regions of 3 and 4 sites) and of the CTA classes
    // of 6 and 7 sites: class k's unit u
    // (= instance * count + position in the class list) owns the D x D row-major complex matrix
    // at warm + warm_off[k] + u D^2 (warm_off[k] < 0: no stored basis for the class)
    float2* warm;
    int64_t warm_off[kClassSlots];
};

// Record `msg` as the thread-local detail returned by lrh_last_error; returns `code`.
int set_last_error(int code, const std::string& msg);

// Kernel attributes (dynamic shared memory limits) for the current device; called once per
// problem creation, outside any stream capture.
cudaError_t prepare_kernels();
cudaError_t prepare_cta_kernels();   // lrh_cta.cu (D = 64, 128, 256)
// Global scratch of the D = 256 pass and certification: complex entries per CTA slot for a
// rotation log of `log_sweeps` sweeps, and the CTAs a launch uses on this device.
int64_t big_slot_elems(int log_sweeps);
// Adjoint of the 6- and 7-site classes (lrh_cta.cu): CTAs of one launch (scratch slots of
// 2 D^2 complex each) and the launch.
cudaError_t vjp_cta_slots(int k, int* slots);
cudaError_t launch_vjp_cta(const DevProblem& P, int k, const int32_t* cls, int32_t count, float2* scratch, int slots,
                           cudaStream_t s);
cudaError_t big_launch_slots(int* slots);
cudaError_t prepare_blk_kernels();   // lrh_block.cu (D = 8, 16, 2x2-block layout)
// D = 8, 16 in the Hermitian 2x2-block layout, `threads` per CTA (64, 128 or 256)
cudaError_t launch_region_pass_blk(const DevProblem& P, const PassIO& io, int k, const int32_t* class_regions,
                                   int32_t class_count, cudaStream_t s, int threads);
constexpr int kShapeBlocks = 4096;   // LRH_SHAPE_BLOCKS
constexpr int kShapeWarp16 = 8192;   // LRH_SHAPE_WARP16
// D = 16 in the 2x2-block layout with one warp per region, `threads` per CTA (64, 128 or 256)
cudaError_t launch_region_pass_w16(const DevProblem& P, const PassIO& io, const int32_t* class_regions,
                                   int32_t class_count, cudaStream_t s, int threads);
cudaError_t launch_region_pass_cta(const DevProblem& P, const PassIO& io, int k, const int32_t* class_regions,
                                   int32_t class_count, cudaStream_t s);
cudaError_t launch_certify_cta(const DevProblem& P, int k, const int32_t* class_regions, int32_t class_count,
                               const float2* msg, cudaStream_t s);

// Launchers (lrh_kernels.cu).  All enqueue on `s` and return the launch status.
cudaError_t launch_region_pass(const DevProblem& P, const PassIO& io, int k, const int32_t* class_regions,
                               int32_t class_count, cudaStream_t s, int block = 128);
// Alg. 2: apply the pending update of iteration t0 + rel into the canonical nu, zeta.
cudaError_t launch_finalize(const DevProblem& P, const PassIO& io, cudaStream_t s);
// Halo exchange of a sharded iteration: copies, for every instance, the 4-entry chunks listed in
// map (>= 0: complex offset in the state arena rho; < 0: ~offset in the partial-trace arena tr)
// into (unpack = 0) or out of (unpack = 1) the packed buffer buf[n_inst][4 n_chunks].
cudaError_t launch_halo_copy(const DevProblem& P, const int64_t* map, int64_t n_chunks, float2* buf, int unpack,
                             cudaStream_t s);
// Alg. 2: t0 += n.
cudaError_t launch_advance(const DevProblem& P, int n, cudaStream_t s);
cudaError_t launch_certify(const DevProblem& P, int k, const int32_t* class_regions,
                           int32_t class_count, const float2* msg, cudaStream_t s);
cudaError_t launch_update(const DevProblem& P, int par, int mode, cudaStream_t s);
cudaError_t launch_reduce(const DevProblem& P, const double* vals, int track_best, cudaStream_t s);
cudaError_t launch_set_state(const DevProblem& P, int par, double theta, double t, int set_theta_t,
                             double beta, double inv_lhat, double alpha, double degen_tol,
                             int variant, int step_rule, int max_sweeps, int cert_sweeps, int cold, cudaStream_t s);
// every stored eigenbasis (n_mats matrices of D x D) set to the identity
cudaError_t launch_warm_identity(float2* warm, int64_t n_mats, int D, cudaStream_t s);
// h32[i] = h64[i] rounded to FP32 (n complex entries)
cudaError_t launch_round_terms(float2* h32, const double2* h64, int64_t n, cudaStream_t s);
cudaError_t launch_copy(float2* dst, const float2* src, int64_t n, cudaStream_t s);

// Adjoint (lrh_vjp.cu): theta_bar per region for the classes, then nu_bar and term cotangents.
cudaError_t prepare_vjp_kernels();
cudaError_t launch_vjp_region(const DevProblem& P, int k, const int32_t* class_regions, int32_t class_count,
                              cudaStream_t s);
cudaError_t launch_vjp_outputs(const DevProblem& P, float2* nu_bar, float2* term_bar, cudaStream_t s);

// update modes
enum : int { UPD_STEP = 0, UPD_GRAD_ONLY = 1 };

// Persistent iteration (lrh_kernels.cu): one cooperative launch for n iterations over up to
// kPersistClasses size classes with k <= 4 (kmax = the largest k, at least 2).  Tiles of class
// c are [tile0[c], tile0[c + 1]); a tile holds persistent_tile_regions(k) regions.
constexpr int kPersistClasses = 4;
struct PersistPlan {
    const int32_t* cls[kPersistClasses];
    int32_t count[kPersistClasses];
    int32_t k[kPersistClasses];
    int64_t tile0[kPersistClasses];
    int64_t tiles;
    int32_t n_classes;
    int32_t n;            // iterations
    int32_t nesterov;     // 1: fused Alg. 2 passes; 0: Alg. 1 iterations
    int32_t par0;         // Alg. 1: parity of the first iteration
    int32_t blk_mask;     // bit k: class k (3 or 4 sites) runs in the 2x2-block layout; bit 5: the
                          // 4-site class in that layout with one warp per region
    unsigned* bar;        // device arrival counter of the grid barrier (zeroed by launch_persistent)
    unsigned expect;      // arrivals per barrier (the grid; set by launch_persistent)
};
int persistent_tile_regions(int k, int32_t blk_mask);
cudaError_t persistent_prepare(int kmax, int* blocks_per_sm);
// One region pass of every class of the plan in one ordinary launch (grid = plan tiles).
cudaError_t launch_class_pass(const DevProblem& P, const PersistPlan& L, int kmax, const PassIO& io, cudaStream_t s);
// unreleased = true (self-test of the bounded wait): every barrier expects one CTA more than the
// grid, so the first barrier never opens and every CTA returns after its wait limit with
// DEV_ERR_TIMEOUT.
cudaError_t launch_persistent(const DevProblem& P, const PersistPlan& L, int kmax, int grid, cudaStream_t s,
                              bool unreleased = false);

}  // namespace lrh
