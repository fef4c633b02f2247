// Allocation-free evaluation of the smoothed pairwise (level-1) dual: lrh_level1_eval_noalloc.
//
// Some callers cannot call cudaMalloc at all: code running inside another runtime's memory
// pool or allocator hook, processes whose device memory is fully reserved up front, or
// embedders that forbid driver allocations after start-up.  They cannot use lrh_create,
// which owns device state.  This entry point computes, from caller-owned device buffers,
// the same region pass + gradient as lrh_evaluate does for an edge/site relaxation, with its
// intermediate data (site accumulators, site Gibbs states, per-region values) held in one
// file-scope __device__ array of fixed size instead of allocated memory.
//
// The scratch array is part of the library image: every GPU that loads the library holds
// it (about 5 MB) until the process exits.  All calls share it and it keeps the contents
// of the last call, so calls whose work overlaps on the GPU (different streams, or
// different host threads without ordering) race with each other and must be serialised by
// the caller.  The first call on a device looks the array's device address up
// (cudaGetSymbolAddress with that device current) and caches it; make that first call
// before any stream capture.
#include "../../include/lrh.h"
#include "lrh_device.cuh"
#include "lrh_internal.cuh"

#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

namespace lrh {
namespace {

constexpr int kNaMaxSites = 65536;    // LRH_NOALLOC_MAX_SITES
constexpr int kNaMaxEdges = 131072;   // LRH_NOALLOC_MAX_EDGES
constexpr int kNaBlock = 128;

// Site sums are taken in a fixed order (ascending edge index), so that repeated calls give
// bit-identical results: the incident edge ends of every site are grouped by a counting sort
// and each site's short list is sorted before its messages are added.
struct NoAllocScratch {
    int32_t start[kNaMaxSites + 1];         // offsets of each site's incident edge ends in `ends`
    int32_t fill[kNaMaxSites];              // per-site counts, then fill cursors
    int32_t ends[2 * kNaMaxEdges];          // incident edge ends t = 2 e + end, grouped by site
    float2 rho_site[kNaMaxSites * 4];       // Gibbs state of every site
    double val[kNaMaxEdges + kNaMaxSites];  // F_beta per edge, then per site
    int32_t bad;                            // an edge endpoint outside [0, n_sites) or a repeated site
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

std::mutex g_scratch_mu;
void* g_scratch_addr[128] = {nullptr};

__device__ __forceinline__ bool na_valid_end(const int32_t* edges, int t, int n_sites) {
    const int site = edges[t];
    return site >= 0 && site < n_sites && edges[t ^ 1] != site;
}

__global__ void na_zero_kernel(NoAllocScratch* S, int n_sites) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_sites) S->fill[i] = 0;
    if (i == 0) S->bad = 0;
}

// incident edge ends per site (endpoints outside [0, n_sites) or repeated are flagged, not used)
__global__ void na_count_kernel(NoAllocScratch* S, const int32_t* __restrict__ edges, int n_edges, int n_sites) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * n_edges) return;
    if (na_valid_end(edges, t, n_sites)) atomicAdd(&S->fill[edges[t]], 1);
    else atomicOr(&S->bad, 1);
}

// exclusive prefix sum of the counts into start[], counts reset to 0 (fill cursors); one block
constexpr int kNaScan = 1024;
__global__ void __launch_bounds__(kNaScan) na_scan_kernel(NoAllocScratch* S, int n_sites) {
    __shared__ int32_t part[kNaScan];
    const int per = (n_sites + kNaScan - 1) / kNaScan;
    const int lo = threadIdx.x * per, hi = min(lo + per, n_sites);
    int32_t acc = 0;
    for (int i = lo; i < hi; ++i) acc += S->fill[i];
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 1; o < kNaScan; o <<= 1) {   // inclusive Hillis-Steele scan of the partial sums
        const int32_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int32_t run = part[threadIdx.x] - acc;
    for (int i = lo; i < hi; ++i) {
        const int32_t c = S->fill[i];
        S->start[i] = run;
        S->fill[i] = 0;
        run += c;
    }
    if (threadIdx.x == kNaScan - 1) S->start[n_sites] = part[kNaScan - 1];
}

__global__ void na_fill_kernel(NoAllocScratch* S, const int32_t* __restrict__ edges, int n_edges, int n_sites) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * n_edges || !na_valid_end(edges, t, n_sites)) return;
    const int site = edges[t];
    S->ends[S->start[site] + atomicAdd(&S->fill[site], 1)] = t;
}

// site Gibbs states: theta_i = h_i + sum of incoming edge messages in ascending edge order, then
// the closed form of a 2 x 2 Hermitian matrix (see region_pass_d2_kernel)
__global__ void na_site_kernel(NoAllocScratch* S, const float2* __restrict__ h_site, const float2* __restrict__ nu,
                               int n_sites, int n_edges, float beta) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_sites) return;
    const int b0 = S->start[i], b1 = S->start[i + 1];
    for (int x = b0 + 1; x < b1; ++x) {   // insertion sort of this site's (short) list
        const int32_t v = S->ends[x];
        int y = x - 1;
        while (y >= b0 && S->ends[y] > v) { S->ends[y + 1] = S->ends[y]; --y; }
        S->ends[y + 1] = v;
    }
    float a = 0.f, br = 0.f, bi = 0.f, d = 0.f;
    if (h_site) { a = h_site[4 * i].x; br = h_site[4 * i + 1].x; bi = h_site[4 * i + 1].y; d = h_site[4 * i + 3].x; }
    for (int x = b0; x < b1; ++x) {
        const float2* m = nu + 4 * S->ends[x];   // nu + 8 e + 4 end
        a += m[0].x; br += m[1].x; bi += m[1].y; d += m[3].x;
    }
    const float m = 0.5f * (a + d), hh = 0.5f * (a - d);
    const float rr = sqrtf(hh * hh + br * br + bi * bi);
    const float kap = rr > 0.f ? tanhf(beta * rr) / rr : beta;
    const float F = (m - rr) - log1pf(expf(-2.0f * beta * rr)) / beta;
    S->rho_site[4 * i + 0] = make_float2(0.5f * (1.f - kap * hh), 0.f);
    S->rho_site[4 * i + 1] = make_float2(-0.5f * kap * br, -0.5f * kap * bi);
    S->rho_site[4 * i + 2] = make_float2(-0.5f * kap * br, 0.5f * kap * bi);
    S->rho_site[4 * i + 3] = make_float2(0.5f * (1.f + kap * hh), 0.f);
    S->val[n_edges + i] = (double)F;
}

// edge Gibbs states (4 lanes per edge, lane-row Jacobi), partial traces and the gradient
// g_{e->first} = rho_first - Tr_second rho_e,  g_{e->second} = rho_second - Tr_first rho_e
__global__ void __launch_bounds__(kNaBlock) na_edge_kernel(NoAllocScratch* S, const int32_t* __restrict__ edges,
                                                           const float2* __restrict__ h_edge,
                                                           const float2* __restrict__ nu, float2* __restrict__ grad,
                                                           int n_edges, int n_sites, float beta) {
    using namespace dev;
    constexpr int D = 4, G = kNaBlock / D;
    __shared__ Rot<float> prm_all[G][D / 2];
    __shared__ float2 Wb_all[G][D * D];
    __shared__ float2 Rb_all[G][D * D];
    __shared__ float pw_all[G][D];
    const int g = threadIdx.x / D, s = threadIdx.x % D;
    const int e = blockIdx.x * G + g;
    const bool valid = e < n_edges;
    float ar[D], ai[D], vr[D], vi[D];
#pragma unroll
    for (int c = 0; c < D; ++c) { ar[c] = 0.f; ai[c] = 0.f; vr[c] = (c == s) ? 1.f : 0.f; vi[c] = 0.f; }
    if (valid) {
        if (h_edge) {
#pragma unroll
            for (int c = 0; c < D; ++c) { const float2 v = h_edge[16 * e + 4 * s + c]; ar[c] = v.x; ai[c] = v.y; }
        }
        const float2* n0 = nu + 8 * e;       // nu_{e->first}: acts on bit 1 of the edge index
        const float2* n1 = nu + 8 * e + 4;   // nu_{e->second}: acts on bit 0
#pragma unroll
        for (int c = 0; c < D; ++c) {
            if (((s ^ c) & 1) == 0) { const float2 m = n0[2 * (s >> 1) + (c >> 1)]; ar[c] -= m.x; ai[c] -= m.y; }
        }
#pragma unroll
        for (int c = 0; c < D; ++c) {
            if (((s ^ c) & 2) == 0) { const float2 m = n1[2 * (s & 1) + (c & 1)]; ar[c] -= m.x; ai[c] -= m.y; }
        }
    }
    float norm2, off2;
    jacobi_lanes<D, float, true>(ar, ai, vr, vi, s, prm_all[g], 15, 1e-12f, norm2, off2);
    float e0, e1;
    pick_pair<D>(ar, s, e0, e1);
    const float lam = (s & 1) ? e1 : e0;
    const float lmin = group_min<D>(lam);
    const float ex = expf(-beta * (lam - lmin));
    const float Z = group_sum<D>(ex);
    const float F = lmin - logf(Z) / beta;
    float* pw = pw_all[g];
    float2* Wb = Wb_all[g];
    float2* Rb = Rb_all[g];
    pw[s] = sqrtf(ex / Z);
    __syncwarp();
#pragma unroll
    for (int c = 0; c < D; ++c) { const float q = pw[c]; Wb[s * D + c] = make_float2(vr[c] * q, vi[c] * q); }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < D; ++j) {
        float accr = 0.f, acci = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const float2 w = Wb[s * D + c], x = Wb[j * D + c];
            accr += w.x * x.x + w.y * x.y;
            acci += w.y * x.x - w.x * x.y;
        }
        Rb[s * D + j] = make_float2(accr, acci);
    }
    __syncwarp();
    float2 fix[D];
#pragma unroll
    for (int j = 0; j < D; ++j) { const float2 up = Rb[j * D + s]; fix[j] = make_float2(up.x, -up.y); }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < D; ++j) {
        if (j < s) Rb[s * D + j] = fix[j];
        if (j == s) Rb[s * D + j].y = 0.f;
    }
    __syncwarp();
    if (valid) {
        // lane s writes entry (a, b) = (s >> 1, s & 1) of both gradient blocks
        const int a = s >> 1, b = s & 1;
        const float2 t0a = Rb[(2 * a + 0) * D + (2 * b + 0)], t0b = Rb[(2 * a + 1) * D + (2 * b + 1)];
        const float2 t1a = Rb[(0 + a) * D + (0 + b)], t1b = Rb[(2 + a) * D + (2 + b)];
        const float qnan = __int_as_float(0x7fc00000);
        if (na_valid_end(edges, 2 * e, n_sites) && na_valid_end(edges, 2 * e + 1, n_sites)) {
            const int f0 = edges[2 * e], f1 = edges[2 * e + 1];
            const float2 r0 = S->rho_site[4 * f0 + s], r1 = S->rho_site[4 * f1 + s];
            grad[8 * e + s] = make_float2(r0.x - (t0a.x + t0b.x), r0.y - (t0a.y + t0b.y));
            grad[8 * e + 4 + s] = make_float2(r1.x - (t1a.x + t1b.x), r1.y - (t1a.y + t1b.y));
        } else {   // a bad endpoint: no site state is read; the outputs say so
            grad[8 * e + s] = make_float2(qnan, qnan);
            grad[8 * e + 4 + s] = make_float2(qnan, qnan);
        }
        if (s == 0) S->val[e] = (double)F;
    }
}

// deterministic FP64 sum of all region values
__global__ void __launch_bounds__(256) na_reduce_kernel(const NoAllocScratch* S, int n, double* out) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) acc += S->val[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = S->bad ? __longlong_as_double(0x7ff8000000000000ll) : sh[0];
}

int scratch_address(NoAllocScratch** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_last_error(LRH_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 128) return set_last_error(LRH_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return set_last_error(LRH_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<NoAllocScratch*>(g_scratch_addr[dev]);
    return LRH_OK;
}

}  // namespace
}  // namespace lrh

extern "C" int lrh_level1_eval_noalloc(int32_t n_sites, int32_t n_edges, const int32_t* edges, const void* h_edge,
                                       const void* h_site, const void* nu, double beta, double* value_out,
                                       void* grad_out, void* stream) {
    using namespace lrh;
    if (n_sites <= 0 || n_edges < 0) return set_last_error(LRH_EINVAL, "n_sites must be > 0 and n_edges >= 0");
    if (n_sites > kNaMaxSites || n_edges > kNaMaxEdges)
        return set_last_error(LRH_EINVAL, "lrh_level1_eval_noalloc handles at most " + std::to_string(kNaMaxSites) +
                                              " sites and " + std::to_string(kNaMaxEdges) + " edges (got " +
                                              std::to_string(n_sites) + ", " + std::to_string(n_edges) + ")");
    if (!(beta > 0.0) || !std::isfinite(beta)) return set_last_error(LRH_EINVAL, "beta must be finite and > 0");
    if (!value_out || (n_edges > 0 && (!edges || !nu || !grad_out)))
        return set_last_error(LRH_EINVAL, "NULL input or output pointer");
    NoAllocScratch* S = nullptr;
    int rc = scratch_address(&S);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const float b = (float)beta;
    const float2* nu2 = static_cast<const float2*>(nu);
    na_zero_kernel<<<(n_sites + 255) / 256, 256, 0, s>>>(S, n_sites);
    if (n_edges > 0) na_count_kernel<<<(2 * n_edges + 255) / 256, 256, 0, s>>>(S, edges, n_edges, n_sites);
    na_scan_kernel<<<1, kNaScan, 0, s>>>(S, n_sites);
    if (n_edges > 0) na_fill_kernel<<<(2 * n_edges + 255) / 256, 256, 0, s>>>(S, edges, n_edges, n_sites);
    na_site_kernel<<<(n_sites + 255) / 256, 256, 0, s>>>(S, static_cast<const float2*>(h_site), nu2, n_sites, n_edges, b);
    if (n_edges > 0) {
        constexpr int G = kNaBlock / 4;
        na_edge_kernel<<<(n_edges + G - 1) / G, kNaBlock, 0, s>>>(S, edges, static_cast<const float2*>(h_edge), nu2,
                                                                  static_cast<float2*>(grad_out), n_edges, n_sites, b);
    }
    na_reduce_kernel<<<1, 256, 0, s>>>(S, n_edges + n_sites, value_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_last_error(LRH_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return LRH_OK;
}
