// CUDA kernels of the message-passing dual solvers (sm_103a).
//
// Region pass (one launch per region-size class k, D = 2^k):
//   assemble theta_e (Sec. 4.2 local augmented Hamiltonian; Alg. 2 extrapolation
//   eta = (1-theta_k) nu + theta_k zeta fused into the message gathers), eigendecompose it
//   in FP32, form the Gibbs state (Sec. 4.1.2) or the normalised ground projector (Alg. 1),
//   store rho_e for the parents' gradients, the partial traces Tr_{e\f} rho_e for every
//   child f, and the per-region value F_beta / lambda_min as a double.
//
// Eigensolver layout for 4 <= D <= 32: a group of D consecutive lanes owns one region.
// Lane s holds row "slot s" of theta (D complex registers) and row s of the eigenvector
// matrix V.  A sweep of the cyclic two-sided complex Jacobi method runs D-1 rounds of the
// round-robin (circle) tournament; in every round the D/2 disjoint pairs are always the
// slot pairs (2k, 2k+1), and the tournament's rotation is applied as a fixed permutation of
// slots: columns move between registers (compile-time indices), rows move between lanes
// (one shuffle per element).  After D-1 rounds the slots are back in natural order.
//   * column rotation A <- A J and V <- V J: lane-local, with (c, w) of all pairs broadcast
//     through shared memory;
//   * row rotation A <- J^H A: each lane gathers the two source rows of its new slot with
//     shuffles, which also performs the tournament's row permutation.
// D = 2 uses the closed form of a 2 x 2 Hermitian matrix.  FP64 is used only by the
// certification pass (lambda_min of theta rebuilt in FP64) and by the bound reduction.
#include "lrh_internal.cuh"
#include "lrh_device.cuh"
#include "lrh_block.cuh"

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>

namespace lrh {

namespace {

constexpr int kBlock = 128;
using namespace dev;

template <int D, int BLOCK>
struct PassSmem {
    static constexpr int kGroups = BLOCK / D;
    static constexpr int LD = D + 2;   // padded row stride (float2) of the W / rho staging: rows of
                                       // different lanes start in different banks, float4 stays aligned
    static constexpr size_t per_group = (D / 2) * sizeof(Rot<float>) + D * sizeof(float) + 2 * D * LD * sizeof(float2);
    static constexpr size_t bytes = kGroups * per_group + 16;
};

// Register budget per lane of the lane-row pass (A and V rows plus the round's temporaries).
template <int D> struct RegCap { static constexpr int v = D == 32 ? 232 : (D == 16 ? 128 : (D == 8 ? 96 : 80)); };

// FP32 region pass for 4 <= D <= 32; BLOCK threads = BLOCK / D regions per CTA (autotuned).
template <int D, int BLOCK>
__device__ __forceinline__ void region_pass_impl(const DevProblem& P, const PassIO& io, const int32_t* __restrict__ cls,
                                                 const int32_t count, const int k, const int64_t tile) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int G = BLOCK / D;
    const int g = threadIdx.x / D;
    const int s = threadIdx.x % D;
    unsigned char* base = smem_raw + g * PassSmem<D, BLOCK>::per_group;
    Rot<float>* prm = reinterpret_cast<Rot<float>*>(base);
    constexpr int LD = PassSmem<D, BLOCK>::LD;
    float2* Wb = reinterpret_cast<float2*>(base + (D / 2) * sizeof(Rot<float>));
    float2* Rb = Wb + D * LD;
    float* pw = reinterpret_cast<float*>(Rb + D * LD);
    __shared__ unsigned long long blk_sweeps, blk_capped;
    if (threadIdx.x == 0) { blk_sweeps = 0ull; blk_capped = 0ull; }

    const int64_t unit = tile * G + g;
    const bool valid = unit < (int64_t)P.n_inst * count;
    const int inst = valid ? (int)(unit / count) : 0;
    // contiguous class of a latency-bound size: the region id without a dependent load
    int r = 0;
    if constexpr (D <= 8) {
        const int cb = P.class_base[D == 4 ? 2 : 3];
        r = valid ? (cb >= 0 ? cb + (int)(unit % count) : cls[unit % count]) : 0;
    } else {
        r = valid ? cls[unit % count] : 0;
    }
    const bool nest = P.st->variant == 1;
    const int max_sweeps = P.st->max_sweeps;
    const Thetas T = pass_thetas(P, io);

    float ar[D], ai[D], vr[D], vi[D];
    RegionInfo R;
    if (valid) {
        if constexpr (D <= 8) {   // uniform class: the region record without a dependent load
            constexpr int KD = D == 4 ? 2 : 3;
            R = ((P.class_uniform >> KD) & 1) ? uniform_region(P.class_first[KD], r - P.class_base[KD], (int64_t)D * D)
                                               : P.reg[r];
        } else {
            R = P.reg[r];
        }
        assemble_row_io<D>(P, R, inst, s, io, T, ar, ai);
    } else {
        R = RegionInfo{-1, -1, 0, 0, 0, 0, 0};
#pragma unroll
        for (int c = 0; c < D; ++c) { ar[c] = 0.f; ai[c] = 0.f; }
    }
#pragma unroll
    for (int c = 0; c < D; ++c) { vr[c] = (c == s) ? 1.f : 0.f; vi[c] = 0.f; }

    float norm2, off2;
    const int sweeps = jacobi_lanes<D, float, true>(ar, ai, vr, vi, s, prm, max_sweeps, 1e-12f, norm2, off2);

    // eigenvalue of slot s, value and state weights
    float e0, e1;
    pick_pair<D>(ar, s, e0, e1);
    const float lam = (s & 1) ? e1 : e0;
    const float lmin = group_min<D>(lam);
    float wgt, F;
    if (nest) {
        const float beta = (float)P.st->beta;
        const float e = expf(-beta * (lam - lmin));
        const float Z = group_sum<D>(e);
        wgt = e / Z;
        F = lmin - logf(Z) / beta;
    } else {
        const float tau = (float)P.st->degen_tol * fmaxf(1.0f, sqrtf(norm2));
        const float in = (lam - lmin <= tau) ? 1.0f : 0.0f;
        const float m = group_sum<D>(in);
        wgt = in / m;
        F = lmin;
    }
    pw[s] = sqrtf(wgt);
    __syncwarp();
    // W = V diag(sqrt(p)); rho = W W^dagger, row s per lane
#pragma unroll
    for (int c = 0; c < D; ++c) { const float q = pw[c]; ar[c] = vr[c] * q; ai[c] = vi[c] * q; }
    {
        float4* wrow = reinterpret_cast<float4*>(Wb + s * LD);
#pragma unroll
        for (int c = 0; c < D / 2; ++c) wrow[c] = make_float4(ar[2 * c], ai[2 * c], ar[2 * c + 1], ai[2 * c + 1]);
    }
    __syncwarp();
    for (int j = 0; j < D; ++j) {
        const float4* wj = reinterpret_cast<const float4*>(Wb + j * LD);
        float accr = 0.f, acci = 0.f;
#pragma unroll
        for (int c = 0; c < D / 2; ++c) {
            const float4 x = wj[c];
            accr += ar[2 * c] * x.x + ai[2 * c] * x.y;
            acci += ai[2 * c] * x.x - ar[2 * c] * x.y;
            accr += ar[2 * c + 1] * x.z + ai[2 * c + 1] * x.w;
            acci += ai[2 * c + 1] * x.z - ar[2 * c + 1] * x.w;
        }
        Rb[s * LD + j] = make_float2(accr, acci);
    }
    __syncwarp();
    // Make rho exactly Hermitian (the two triangles come from differently rounded sums):
    // row s keeps its upper part, takes the conjugate of the upper part for j < s, and a
    // real diagonal.  Exactly Hermitian states keep every message exactly Hermitian.
    {
        float2 fix[D];
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const float2 up = Rb[j * LD + s];
            fix[j] = make_float2(up.x, -up.y);
        }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < D; ++j) {
            if (j < s) Rb[s * LD + j] = fix[j];
            if (j == s) Rb[s * LD + j].y = 0.f;
        }
    }
    __syncwarp();
    if (valid) {
        if (R.rho_off >= 0) {
            float4* dst = reinterpret_cast<float4*>(io.rho_out + (int64_t)inst * P.rho_elems + R.rho_off + (int64_t)s * D);
            const float4* srcr = reinterpret_cast<const float4*>(Rb + s * LD);
#pragma unroll
            for (int c = 0; c < D / 2; ++c) dst[c] = srcr[c];
        }
        float2* trb = io.tr_out + (int64_t)inst * P.msg_elems;
        for (int q = R.child_begin; q < R.child_end; ++q) {
            const PairInfo pi = P.child_info[q];
            const int M = pi.mask;
            const int Mc = (D - 1) & ~M;
            const int kf = pi.kf;
            const int Df = 1 << kf;
            const int nrest = D >> kf;
            for (int idx = s; idx < Df * Df; idx += D) {
                const int ra = pdep_bits(idx >> kf, M);
                const int rb = pdep_bits(idx & (Df - 1), M);
                float accr = 0.f, acci = 0.f;
                int x = 0;   // pdep(c, Mc) for c = 0, 1, ...: the submasks of Mc in increasing order
                for (int c = 0; c < nrest; ++c) {
                    const float2 v = Rb[(ra | x) * LD + (rb | x)];
                    accr += v.x;
                    acci += v.y;
                    x = ((x | ~Mc) + 1) & Mc;
                }
                trb[pi.off + idx] = make_float2(accr, acci);
            }
        }
        if (s == 0) {
            P.val[(int64_t)inst * P.n_regions + r] = (double)F;
            if (!isfinite(F)) atomicOr(P.err, DEV_ERR_NUMERIC);
        }
    }
    // sweep accounting (regions x sweeps, regions stopped by the sweep cap), one global atomic per block
    __syncthreads();
    if (valid && s == 0) {
        atomicAdd(&blk_sweeps, (unsigned long long)sweeps);
        if (off2 > 1e-12f * norm2) atomicAdd(&blk_capped, 1ull);
    }
    __syncthreads();
    if (threadIdx.x == 0 && blk_sweeps) atomicAdd(&P.sweeps[k], blk_sweeps);
    if (threadIdx.x == 0 && blk_capped) atomicAdd(&P.capped[k], blk_capped);
}

template <int D, int BLOCK>
__global__ void __launch_bounds__(BLOCK) __maxnreg__(RegCap<D>::v) region_pass_kernel(const DevProblem P, const PassIO io,
                                                                                       const int32_t* __restrict__ cls,
                                                                                       const int32_t count, const int k) {
    if (io.writer && blockIdx.x == 0 && threadIdx.x == 0) advance_theta(P, io);
    region_pass_impl<D, BLOCK>(P, io, cls, count, k, blockIdx.x);
}

// D = 32 keeps ptxas's own register heuristic (explicit caps made it spill).
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) region_pass_kernel32(const DevProblem P, const PassIO io,
                                                              const int32_t* __restrict__ cls, const int32_t count,
                                                              const int k) {
    if (io.writer && blockIdx.x == 0 && threadIdx.x == 0) advance_theta(P, io);
    region_pass_impl<32, BLOCK>(P, io, cls, count, k, blockIdx.x);
}

// D = 2 closed form, one thread per region.  theta = m I + K, K = [[hh, b], [conj(b), -hh]],
// K^2 = r^2 I with r = sqrt(hh^2 + |b|^2): lambda = m -+ r,
// Gibbs state (1/2)(I - tanh(beta r) K / r), F_beta = m - r - log(1 + e^{-2 beta r}) / beta,
// ground projector (1/2)(I - K / r), or I/2 when 2r is within the degeneracy tolerance.
__device__ __forceinline__ void region_d2_unit(const DevProblem& P, const PassIO& io, const Thetas& T,
                                               const int32_t* __restrict__ cls, const int32_t count, const int64_t unit) {
    if (unit >= (int64_t)P.n_inst * count) return;
    const int inst = (int)(unit / count);
    const int r = P.class_base[1] >= 0 ? P.class_base[1] + (int)(unit % count) : cls[unit % count];
    const bool nest = P.st->variant == 1;
    const RegionInfo R = ((P.class_uniform >> 1) & 1) ? uniform_region(P.class_first[1], r - P.class_base[1], 4) : P.reg[r];
    float a = 0.f, d = 0.f, br = 0.f, bi = 0.f;
    if (R.h_off >= 0) {
        const float2* h = P.h32 + (int64_t)inst * P.h_elems + R.h_off;
        a = h[0].x; br = h[1].x; bi = h[1].y; d = h[3].x;
    }
    const int64_t mbase = (int64_t)inst * P.msg_elems;
    const int64_t rbase = (int64_t)inst * P.rho_elems;
    for (int q = R.parent_begin; q < R.parent_end; ++q) {
        const PairInfo pi = P.parent_info[q];
        const float4 m01 = pass_entry2(io, T, mbase + pi.off, rbase + R.rho_off, true);
        const float4 m23 = pass_entry2(io, T, mbase + pi.off + 2, rbase + R.rho_off + 2, true);
        a += m01.x; br += m01.z; bi += m01.w; d += m23.z;
    }
    // children of a one-site region do not exist (no proper non-empty subset)
    const float m = 0.5f * (a + d);
    const float hh = 0.5f * (a - d);
    const float rr = sqrtf(hh * hh + br * br + bi * bi);
    const float lmin = m - rr;
    float kap, F;
    if (nest) {
        const float beta = (float)P.st->beta;
        kap = rr > 0.f ? tanhf(beta * rr) / rr : beta;
        F = lmin - log1pf(expf(-2.0f * beta * rr)) / beta;
    } else {
        const float nrm = sqrtf(a * a + d * d + 2.f * (br * br + bi * bi));
        const float tau = (float)P.st->degen_tol * fmaxf(1.0f, nrm);
        kap = (2.f * rr > tau) ? 1.0f / rr : 0.0f;
        F = lmin;
    }
    if (R.rho_off >= 0) {
        float4* dst = reinterpret_cast<float4*>(io.rho_out + (int64_t)inst * P.rho_elems + R.rho_off);
        dst[0] = make_float4(0.5f * (1.f - kap * hh), 0.f, -0.5f * kap * br, -0.5f * kap * bi);
        dst[1] = make_float4(-0.5f * kap * br, 0.5f * kap * bi, 0.5f * (1.f + kap * hh), 0.f);
    }
    P.val[(int64_t)inst * P.n_regions + r] = (double)F;
    if (!isfinite(F)) atomicOr(P.err, DEV_ERR_NUMERIC);
}

__global__ void __launch_bounds__(256) region_pass_d2_kernel(const DevProblem P, const PassIO io,
                                                            const int32_t* __restrict__ cls, const int32_t count) {
    const Thetas T = pass_thetas(P, io);
    if (io.writer && blockIdx.x == 0 && threadIdx.x == 0) advance_theta(P, io);
    region_d2_unit(P, io, T, cls, count, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// 4 x 4 regions, one thread per region: the whole cyclic Jacobi runs in registers with
// compile-time indices (six rotations per sweep, in the two-pair rounds (0,1)(2,3),
// (0,2)(1,3), (0,3)(1,2)), so the only dependencies are ALU latencies.  Same inputs,
// outputs and arithmetic conventions as region_pass_kernel<4>.
__device__ __forceinline__ void t4_rotate(float (&ar)[4][4], float (&ai)[4][4], float (&vr)[4][4], float (&vi)[4][4],
                                          int p, int q) {
    float c, wr, wi;
    rot_params(ar[p][p], ar[q][q], ar[p][q], ai[p][q], c, wr, wi);
#pragma unroll
    for (int r = 0; r < 4; ++r) {   // A <- A J  (columns p, q)
        mix_cols(ar[r][p], ai[r][p], ar[r][q], ai[r][q], c, wr, wi);
        mix_cols(vr[r][p], vi[r][p], vr[r][q], vi[r][q], c, wr, wi);
    }
#pragma unroll
    for (int col = 0; col < 4; ++col) {   // A <- J^H A  (rows p, q): y_p' = c y_p + w y_q, y_q' = -conj(w) y_p + c y_q
        const float ypr = ar[p][col], ypi = ai[p][col], yqr = ar[q][col], yqi = ai[q][col];
        ar[p][col] = c * ypr + (wr * yqr - wi * yqi);
        ai[p][col] = c * ypi + (wr * yqi + wi * yqr);
        ar[q][col] = c * yqr - (wr * ypr + wi * ypi);
        ai[q][col] = c * yqi - (wr * ypi - wi * ypr);
    }
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) region_pass_t4_kernel(const DevProblem P, const PassIO io,
                                                               const int32_t* __restrict__ cls, const int32_t count,
                                                               const int k) {
    __shared__ unsigned long long blk_sweeps, blk_capped;
    if (threadIdx.x == 0) { blk_sweeps = 0ull; blk_capped = 0ull; }
    const Thetas T = pass_thetas(P, io);
    if (io.writer && blockIdx.x == 0 && threadIdx.x == 0) advance_theta(P, io);
    __syncthreads();
    const int64_t unit = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
    int sweeps = 0;
    if (unit < (int64_t)P.n_inst * count) {
        const int inst = (int)(unit / count);
        const int r = P.class_base[2] >= 0 ? P.class_base[2] + (int)(unit % count) : cls[unit % count];
        const RegionInfo R = P.reg[r];
        const bool nest = P.st->variant == 1;
        float ar[4][4], ai[4][4], vr[4][4], vi[4][4];
        if (R.h_off >= 0) {
            const float4* h = reinterpret_cast<const float4*>(P.h32 + (int64_t)inst * P.h_elems + R.h_off);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const float4 v = h[2 * i + j];
                    ar[i][2 * j] = v.x; ai[i][2 * j] = v.y; ar[i][2 * j + 1] = v.z; ai[i][2 * j + 1] = v.w;
                }
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) { ar[i][j] = 0.f; ai[i][j] = 0.f; }
        }
        const int64_t mbase = (int64_t)inst * P.msg_elems;
        const int64_t rbase = (int64_t)inst * P.rho_elems;
        // children of a two-site region are its sites: mask 2 = first site (nu (x) 1), mask 1 = second (1 (x) nu)
        for (int q = R.child_begin; q < R.child_end; ++q) {
            const PairInfo pi = P.child_info[q];
            float2 m[2][2];
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    const int x = 2 * a + b;
                    m[a][b] = pass_entry(io, T, mbase + pi.off + x, rbase + pi.child_rho + x, false);
                }
            if (pi.mask == 2) {   // nu (x) 1
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int b = 0; b < 2; ++b)
#pragma unroll
                        for (int o = 0; o < 2; ++o) { ar[2 * a + o][2 * b + o] -= m[a][b].x; ai[2 * a + o][2 * b + o] -= m[a][b].y; }
            } else {              // 1 (x) nu
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int b = 0; b < 2; ++b)
#pragma unroll
                        for (int o = 0; o < 2; ++o) { ar[2 * o + a][2 * o + b] -= m[a][b].x; ai[2 * o + a][2 * o + b] -= m[a][b].y; }
            }
        }
        for (int q = R.parent_begin; q < R.parent_end; ++q) {
            const PairInfo pi = P.parent_info[q];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; j += 2) {
                    const int x = 4 * i + j;
                    const float4 m = pass_entry2(io, T, mbase + pi.off + x, rbase + R.rho_off + x, true);
                    ar[i][j] += m.x; ai[i][j] += m.y; ar[i][j + 1] += m.z; ai[i][j + 1] += m.w;
                }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) { vr[i][j] = (i == j) ? 1.f : 0.f; vi[i][j] = 0.f; }
        float n2 = 0.f;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) n2 += ar[i][j] * ar[i][j] + ai[i][j] * ai[i][j];
        const float thresh = 1e-12f * n2;
        const int max_sweeps = P.st->max_sweeps;
        float off = 0.f;
        for (;;) {
            off = 0.f;
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) off += (i == j) ? 0.f : ar[i][j] * ar[i][j] + ai[i][j] * ai[i][j];
            if (off <= thresh || sweeps >= max_sweeps) break;
            ++sweeps;
            t4_rotate(ar, ai, vr, vi, 0, 1);
            t4_rotate(ar, ai, vr, vi, 2, 3);
            t4_rotate(ar, ai, vr, vi, 0, 2);
            t4_rotate(ar, ai, vr, vi, 1, 3);
            t4_rotate(ar, ai, vr, vi, 0, 3);
            t4_rotate(ar, ai, vr, vi, 1, 2);
        }
        float lam[4], w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) lam[i] = ar[i][i];
        const float lmin = fminf(fminf(lam[0], lam[1]), fminf(lam[2], lam[3]));
        float F;
        if (nest) {
            const float beta = (float)P.st->beta;
            float Z = 0.f;
#pragma unroll
            for (int i = 0; i < 4; ++i) { w[i] = expf(-beta * (lam[i] - lmin)); Z += w[i]; }
#pragma unroll
            for (int i = 0; i < 4; ++i) w[i] /= Z;
            F = lmin - logf(Z) / beta;
        } else {
            const float tau = (float)P.st->degen_tol * fmaxf(1.0f, sqrtf(n2));
            float m = 0.f;
#pragma unroll
            for (int i = 0; i < 4; ++i) { w[i] = (lam[i] - lmin <= tau) ? 1.f : 0.f; m += w[i]; }
#pragma unroll
            for (int i = 0; i < 4; ++i) w[i] /= m;
            F = lmin;
        }
        // rho = V diag(w) V^dagger, upper triangle computed, lower = conjugate, real diagonal
        float rr[4][4], ri[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = i; j < 4; ++j) {
                float sr = 0.f, si = 0.f;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float xr = w[c] * vr[j][c], xi = w[c] * vi[j][c];
                    sr += vr[i][c] * xr + vi[i][c] * xi;
                    si += vi[i][c] * xr - vr[i][c] * xi;
                }
                rr[i][j] = sr; ri[i][j] = (i == j) ? 0.f : si;
                rr[j][i] = sr; ri[j][i] = (i == j) ? 0.f : -si;
            }
        if (R.rho_off >= 0) {
            float4* dst = reinterpret_cast<float4*>(io.rho_out + rbase + R.rho_off);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j)
                    dst[2 * i + j] = make_float4(rr[i][2 * j], ri[i][2 * j], rr[i][2 * j + 1], ri[i][2 * j + 1]);
        }
        float2* trb = io.tr_out + mbase;
        for (int q = R.child_begin; q < R.child_end; ++q) {
            const PairInfo pi = P.child_info[q];
            float2 tt[2][2];
            if (pi.mask == 2) {   // keep the first site: trace out the second
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int b = 0; b < 2; ++b)
                        tt[a][b] = make_float2(rr[2 * a][2 * b] + rr[2 * a + 1][2 * b + 1], ri[2 * a][2 * b] + ri[2 * a + 1][2 * b + 1]);
            } else {              // keep the second site
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int b = 0; b < 2; ++b)
                        tt[a][b] = make_float2(rr[a][b] + rr[2 + a][2 + b], ri[a][b] + ri[2 + a][2 + b]);
            }
            float4* tdst = reinterpret_cast<float4*>(trb + pi.off);
            tdst[0] = make_float4(tt[0][0].x, tt[0][0].y, tt[0][1].x, tt[0][1].y);
            tdst[1] = make_float4(tt[1][0].x, tt[1][0].y, tt[1][1].x, tt[1][1].y);
        }
        P.val[(int64_t)inst * P.n_regions + r] = (double)F;
        if (!isfinite(F)) atomicOr(P.err, DEV_ERR_NUMERIC);
        atomicAdd(&blk_sweeps, (unsigned long long)sweeps);
        if (off > thresh) atomicAdd(&blk_capped, 1ull);
    }
    __syncthreads();
    if (threadIdx.x == 0 && blk_sweeps) atomicAdd(&P.sweeps[k], blk_sweeps);
    if (threadIdx.x == 0 && blk_capped) atomicAdd(&P.capped[k], blk_capped);
}

// ---------------------------------------------------------------- FP64 certification
template <int D>
struct CertSmem {
    static constexpr int kGroups = kBlock / D;
    static constexpr size_t bytes = kGroups * (D / 2) * sizeof(Rot<double>) + 16;
};

template <int D>
__global__ void __launch_bounds__(kBlock) certify_kernel(const DevProblem P, const int32_t* __restrict__ cls,
                                                         const int32_t count, const float2* __restrict__ msg) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int G = kBlock / D;
    const int g = threadIdx.x / D;
    const int s = threadIdx.x % D;
    Rot<double>* prm = reinterpret_cast<Rot<double>*>(smem_raw) + g * (D / 2);
    const int64_t unit = (int64_t)blockIdx.x * G + g;
    const bool valid = unit < (int64_t)P.n_inst * count;
    const int inst = valid ? (int)(unit / count) : 0;
    const int r = valid ? cls[unit % count] : 0;
    double ar[D], ai[D], vr[D], vi[D];
    if (valid) {
        const RegionInfo R = P.reg[r];
        assemble_row<D, double>(P, R, inst, s, msg, nullptr, 0.0f, true, ar, ai);
    } else {
#pragma unroll
        for (int c = 0; c < D; ++c) { ar[c] = 0.0; ai[c] = 0.0; }
    }
    double norm2, off2;
    jacobi_lanes<D, double, false>(ar, ai, vr, vi, s, prm, P.st->cert_sweeps, 1e-28, norm2, off2);
    double e0, e1;
    pick_pair<D>(ar, s, e0, e1);
    const double lam = (s & 1) ? e1 : e0;
    // Weyl: the rotated matrix is diag(a) + E with ||E||_2 <= ||E||_F = sqrt(off2), so
    // lambda_min >= min_i a_ii - sqrt(off2): a lower bound even when the sweep cap stopped the
    // iteration (then flagged); at convergence the correction is below 1e-14 ||theta||_F.
    const double lmin = group_min<D>(lam) - sqrt(off2);
    if (valid && s == 0) {
        P.val64[(int64_t)inst * P.n_regions + r] = lmin;
        if (!isfinite(lmin)) atomicOr(P.err, DEV_ERR_NUMERIC);
        if (off2 > 1e-28 * norm2) atomicOr(P.err, DEV_ERR_NOCONV);
    }
}

__global__ void certify_d2_kernel(const DevProblem P, const int32_t* __restrict__ cls, const int32_t count,
                                  const float2* __restrict__ msg) {
    const int64_t unit = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (unit >= (int64_t)P.n_inst * count) return;
    const int inst = (int)(unit / count);
    const int r = cls[unit % count];
    const RegionInfo R = P.reg[r];
    double a = 0, d = 0, br = 0, bi = 0;
    if (R.h_off >= 0) {
        const double2* h = P.h64 + (int64_t)inst * P.h_elems + R.h_off;
        a = h[0].x; br = h[1].x; bi = h[1].y; d = h[3].x;
    }
    const int64_t mbase = (int64_t)inst * P.msg_elems;
    for (int q = R.parent_begin; q < R.parent_end; ++q) {
        const PairInfo pi = P.parent_info[q];
        const float2* nb = msg + mbase + pi.off;
        a += (double)nb[0].x; br += (double)nb[1].x; bi += (double)nb[1].y; d += (double)nb[3].x;
    }
    const double m = 0.5 * (a + d), hh = 0.5 * (a - d);
    const double lmin = m - sqrt(hh * hh + br * br + bi * bi);
    P.val64[(int64_t)inst * P.n_regions + r] = lmin;
    if (!isfinite(lmin)) atomicOr(P.err, DEV_ERR_NUMERIC);
}

// ---------------------------------------------------------------- message update
// One thread per two consecutive complex entries of one instance's message array (every
// block holds D_f^2 >= 4 entries, so the two never straddle pairs).
// Alg. 1 update (and the gradient-only mode of lrh_evaluate), one thread per two consecutive
// complex entries of one instance's message array (every block holds D_f^2 >= 4 entries, so
// the two never straddle pairs): g = rho_f - Tr_{e\f} rho_e; nu += alpha_t g, with nu_best
// copied first when the previous pass set a new best q.
__device__ __forceinline__ void update_elem(const DevProblem& P, const int par, const int mode, const int64_t tid) {
    const int64_t halfm = P.msg_elems >> 1;
    const double td = P.st->t[par];
    if (tid == 0 && mode == UPD_STEP) P.st->t[par ^ 1] = td + 1.0;
    if (tid >= (int64_t)P.n_inst * halfm) return;
    const int inst = (int)(tid / halfm);
    const int64_t e = (tid % halfm) * 2;
    const int64_t mi = (int64_t)inst * P.msg_elems + e;
    const float4 rf = *reinterpret_cast<const float4*>(P.rho + (int64_t)inst * P.rho_elems + P.chunk_rho[e >> 2] + e);
    const float4 tv = *reinterpret_cast<const float4*>(P.tr + mi);
    const float4 gv = make_float4(rf.x - tv.x, rf.y - tv.y, rf.z - tv.z, rf.w - tv.w);
    if (mode == UPD_GRAD_ONLY) {
        *reinterpret_cast<float4*>(P.grad + mi) = gv;
        return;
    }
    float4 nv = *reinterpret_cast<const float4*>(P.nu + mi);
    if (P.best_flag[inst]) *reinterpret_cast<float4*>(P.nu_best + mi) = nv;
    const double a0 = P.st->alpha;
    const float alpha = (float)(P.st->step_rule == 1 ? a0 / sqrt(td + 1.0) : a0);
    nv.x = fmaf(alpha, gv.x, nv.x); nv.y = fmaf(alpha, gv.y, nv.y);
    nv.z = fmaf(alpha, gv.z, nv.z); nv.w = fmaf(alpha, gv.w, nv.w);
    if (!(isfinite(nv.x) && isfinite(nv.y) && isfinite(nv.z) && isfinite(nv.w))) atomicOr(P.err, DEV_ERR_NUMERIC);
    *reinterpret_cast<float4*>(P.nu + mi) = nv;
}

__global__ void update_kernel(const DevProblem P, const int par, const int mode) {
    update_elem(P, par, mode, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// Alg. 2: the pending update of iteration t = t0 + io.rel (its states in io.rho_in / tr_in, its
// multipliers in io.nu_in / zeta_in) written to io.nu_out / zeta_out.
__global__ void finalize_kernel(const DevProblem P, const PassIO io) {
    const int64_t halfm = P.msg_elems >> 1;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (int64_t)P.n_inst * halfm) return;
    const long long t = P.st->t0 + io.rel;
    const double thd = P.st->th3[t % 3];
    const float th = (float)thd;
    const float kz = (float)(P.st->inv_lhat / thd);
    const int inst = (int)(tid / halfm);
    const int64_t e = (tid % halfm) * 2;
    const int64_t mi = (int64_t)inst * P.msg_elems + e;
    const int64_t ri = (int64_t)inst * P.rho_elems + P.chunk_rho[e >> 2] + e;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        float2 n = io.nu_in[mi + j], z = io.zeta_in[mi + j];
        const float2 r = io.rho_in[ri + j], tv = io.tr_in[mi + j];
        nesterov_update(n, z, r.x - tv.x, r.y - tv.y, th, kz);
        if (!(isfinite(n.x) && isfinite(n.y) && isfinite(z.x) && isfinite(z.y))) atomicOr(P.err, DEV_ERR_NUMERIC);
        io.nu_out[mi + j] = n;
        io.zeta_out[mi + j] = z;
    }
}

// Halo exchange of a sharded iteration (see launch_halo_copy): one thread per two complex entries
// (16 bytes; chunk offsets are multiples of 4 entries, the buffer is 16-byte aligned).
__global__ void halo_copy_kernel(const DevProblem P, const int64_t* __restrict__ map, const int64_t n_chunks,
                                 float2* __restrict__ buf, const int unpack) {
    const int64_t per = 2 * n_chunks;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (int64_t)P.n_inst * per) return;
    const int64_t inst = tid / per, u = tid % per;
    const int64_t m = map[u >> 1];
    const int64_t j = (u & 1) * 2;
    float2* arena = m >= 0 ? P.rho + inst * P.rho_elems + m : P.tr + inst * P.msg_elems + ~m;
    float4* a = reinterpret_cast<float4*>(arena + j);
    float4* b = reinterpret_cast<float4*>(buf + inst * 4 * n_chunks + 2 * u);
    if (unpack) *a = *b; else *b = *a;
}

__global__ void advance_kernel(IterState* st, int n) { st->t0 += n; }

// Deterministic per-instance FP64 sum of per-region values (fixed strided partial sums and a
// fixed tree), with optional Alg. 1 best-so-far tracking.
constexpr int kReduce = 256;
// kReduce fixed strided partial sums and a fixed tree, computed by NT <= kReduce threads (each
// thread takes the partial-sum slots vt = threadIdx.x + NT j): the same additions in the same
// order for any NT.  The caller synchronises before reusing sh.
template <int NT>
__device__ __forceinline__ void reduce_instance(const DevProblem& P, const double* __restrict__ vals, const int track_best,
                                                const int inst, double* sh) {
    const double* v = vals + (int64_t)inst * P.n_regions;
    for (int vt = threadIdx.x; vt < kReduce; vt += NT) {
        double acc = 0.0;
        for (int i = vt; i < P.n_regions; i += kReduce) acc += v[i];
        sh[vt] = acc;
    }
    __syncthreads();
    for (int w = kReduce / 2; w > 0; w >>= 1) {
        for (int vt = threadIdx.x; vt < w; vt += NT) sh[vt] += sh[vt + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double q = sh[0];
        P.q_sum[inst] = q;
        if (track_best) {
            const int better = q > P.q_best[inst];
            P.best_flag[inst] = better;
            if (better) P.q_best[inst] = q;
        }
    }
}

__global__ void __launch_bounds__(kReduce) reduce_kernel(const DevProblem P, const double* __restrict__ vals,
                                                        const int track_best) {
    __shared__ double sh[kReduce];
    reduce_instance<kReduce>(P, vals, track_best, blockIdx.x, sh);
}

__global__ void set_state_kernel(IterState* st, int par, double theta, double t, int set_theta_t, double beta,
                                 double inv_lhat, double alpha, double degen_tol, int variant, int step_rule,
                                 int max_sweeps, int cert_sweeps, int cold) {
    if (set_theta_t) {
        st->theta[par] = theta;
        st->t[par] = t;
        st->t0 = 0;
        st->th3[0] = theta;
    }
    st->beta = beta;
    st->inv_lhat = inv_lhat;
    st->alpha = alpha;
    st->degen_tol = degen_tol;
    st->variant = variant;
    st->step_rule = step_rule;
    st->max_sweeps = max_sweeps;
    st->cert_sweeps = cert_sweeps;
    st->cold = cold;
}

__global__ void warm_identity_kernel(float4* w, int64_t n_pairs_total, int D) {
    // entries 2j, 2j+1 of the flattened matrices (D even): (i, c) and (i, c + 1)
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t per = (int64_t)D * D / 2;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_pairs_total; j += stride) {
        const int64_t e = 2 * (j % per);
        const int64_t i = e / D, c = e % D;
        w[j] = make_float4(i == c ? 1.f : 0.f, 0.f, i == c + 1 ? 1.f : 0.f, 0.f);
    }
}

// ---------------------------------------------------------------------------------------------
// Persistent iteration: one cooperative launch (every block resident) runs n iterations over
// all size classes k <= KMAX, with a grid-wide barrier where the graph path has a launch
// boundary.  Per pass, the tiles of all classes (kBlock / D regions of one class per tile;
// kBlock regions for D = 2) are dealt to the blocks round-robin; the per-region code is the
// same as in the per-class kernels, so the results are bit-identical to the graph path.
//   Alg. 2: n fused passes (the PassIO sequence of the graph path), one barrier after each;
//           the caller finalises the last pending update.
//   Alg. 1: pass, barrier, per-instance reduction with best tracking, barrier, message update,
//           barrier.
// ---------------------------------------------------------------------------------------------
constexpr unsigned long long kBarrierLimitNs = 1000000000ull;   // one second per wait

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned atom_add_release(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Grid-wide barrier on one monotonic arrival counter (zeroed before the launch): a CTA adds 1
// with release semantics and waits, with acquire loads, until the counter reaches the end of
// its group of `expect` arrivals.  No reset and no second word, so the last arrival needs no
// extra round trip.  A wait longer than kBarrierLimitNs, or one that sees another CTA's timeout
// (checked every 256 polls), raises DEV_ERR_TIMEOUT and returns false; the caller then returns.
__device__ __forceinline__ bool grid_sync(int32_t* err, unsigned* bar, unsigned expect) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int good = 1;
        const unsigned old = atom_add_release(bar, 1u);
        const unsigned target = (old / expect + 1u) * expect;
        const unsigned long long t0 = global_ns();
        for (unsigned poll = 1; (int)(ld_acquire_u32(bar) - target) < 0; ++poll) {
            if ((poll & 255u) == 0 &&
                ((ld_acquire_u32(reinterpret_cast<const unsigned*>(err)) & DEV_ERR_TIMEOUT) ||
                 global_ns() - t0 > kBarrierLimitNs)) {
                atomicOr(err, DEV_ERR_TIMEOUT);
                good = 0;
                break;
            }
        }
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// PassIO of fused pass j of an n-pass Alg. 2 step: buffers A (nu, zeta), B (nu_b, zeta_b),
// X (rho, tr), Y (rho_b, tr_b); pass j reads A when j is 0 or odd, else B, applies the pending
// update of pass j - 1 (states from X when j is odd, Y when even) into B (odd j) or A (even j),
// and writes its states to X (even j) or Y (odd j).
__device__ __forceinline__ PassIO nesterov_io(const DevProblem& P, const int j) {
    PassIO io{};
    io.rel = j;
    io.writer = 1;
    io.pending = j > 0;
    const bool odd = (j & 1) != 0;
    io.nu_in = (odd || j == 0) ? P.nu : P.nu_b;
    io.zeta_in = (odd || j == 0) ? P.zeta : P.zeta_b;
    if (j > 0) {
        io.rho_in = odd ? P.rho : P.rho_b;
        io.tr_in = odd ? P.tr : P.tr_b;
        io.nu_out = odd ? P.nu_b : P.nu;
        io.zeta_out = odd ? P.zeta_b : P.zeta;
    }
    io.rho_out = odd ? P.rho_b : P.rho;
    io.tr_out = odd ? P.tr_b : P.tr;
    return io;
}

// Register budget of the persistent kernel (its tile loop keeps the pass's PassIO and the plan
// live around the per-region code): no spills up to k = 3; a small one at k = 4.
template <int KMAX> struct PersistCap { static constexpr int v = KMAX == 2 ? 96 : (KMAX == 3 ? 128 : 168); };

// One tile of a pass over all classes of a plan: 128 / D regions of class k (128 for k = 1),
// with the per-region code of the per-class kernels.
template <int KMAX>
__device__ __forceinline__ void plan_tile(const DevProblem& P, const PersistPlan& L, const PassIO& io, const Thetas& T,
                                          const int64_t tile) {
    // class of this tile, with compile-time indices into the plan (no local copy of it)
    int k = L.k[0];
    const int32_t* cls = L.cls[0];
    int32_t count = L.count[0];
    int64_t first = L.tile0[0];
#pragma unroll
    for (int q = 1; q < kPersistClasses; ++q)
        if (q < L.n_classes && tile >= L.tile0[q]) { k = L.k[q]; cls = L.cls[q]; count = L.count[q]; first = L.tile0[q]; }
    const int64_t lt = tile - first;
    if (k == 1) {
        region_d2_unit(P, io, T, cls, count, lt * kBlock + threadIdx.x);
    } else if (k == 2) {
        region_pass_impl<4, kBlock>(P, io, cls, count, 2, lt);
    } else if (k == 3) {
        if constexpr (KMAX >= 3) {
            if ((L.blk_mask >> 3) & 1) blk::region_pass_blk_impl<8, kBlock>(P, io, cls, count, 3, lt);
            else region_pass_impl<8, kBlock>(P, io, cls, count, 3, lt);
        }
    } else {
        if constexpr (KMAX >= 4) {
            if ((L.blk_mask >> 5) & 1) blk::region_pass_w16_impl<kBlock>(P, io, cls, count, 4, lt);
            else if ((L.blk_mask >> 4) & 1) blk::region_pass_blk_impl<16, kBlock>(P, io, cls, count, 4, lt);
            else region_pass_impl<16, kBlock>(P, io, cls, count, 4, lt);
        }
    }
}

// One region pass of every class in one ordinary launch (one CTA per tile): the alternative to
// one launch per class on forked streams; same per-region code, same results.
template <int KMAX>
__global__ void __launch_bounds__(kBlock) __maxnreg__(PersistCap<KMAX>::v)
    class_pass_kernel(const DevProblem P, const PersistPlan L, const PassIO io) {
    if (io.writer && blockIdx.x == 0 && threadIdx.x == 0) advance_theta(P, io);
    const Thetas T = pass_thetas(P, io);
    plan_tile<KMAX>(P, L, io, T, blockIdx.x);
}

template <int KMAX>
__global__ void __launch_bounds__(kBlock) __maxnreg__(PersistCap<KMAX>::v)
    persist_kernel(const DevProblem P, const PersistPlan L) {
    __shared__ double red[kReduce];
    for (int j = 0; j < L.n; ++j) {
        PassIO io{};
        if (L.nesterov) {
            io = nesterov_io(P, j);
            if (blockIdx.x == 0 && threadIdx.x == 0) advance_theta(P, io);
        } else {
            io.nu_in = P.nu;
            io.rho_out = P.rho;
            io.tr_out = P.tr;
        }
        const Thetas T = pass_thetas(P, io);
        for (int64_t tile = blockIdx.x; tile < L.tiles; tile += gridDim.x) plan_tile<KMAX>(P, L, io, T, tile);
        if (!grid_sync(P.err, L.bar, L.expect)) return;
        if (!L.nesterov) {
            const int par = (L.par0 + j) & 1;
            for (int inst = blockIdx.x; inst < P.n_inst; inst += gridDim.x) {
                reduce_instance<kBlock>(P, P.val, 1, inst, red);
                __syncthreads();
            }
            if (!grid_sync(P.err, L.bar, L.expect)) return;
            int64_t nel = (int64_t)P.n_inst * (P.msg_elems >> 1);
            if (nel < 1) nel = 1;   // element 0 also advances the iteration counter
            for (int64_t tid = (int64_t)blockIdx.x * kBlock + threadIdx.x; tid < nel; tid += (int64_t)gridDim.x * kBlock)
                update_elem(P, par, UPD_STEP, tid);
            if (!grid_sync(P.err, L.bar, L.expect)) return;
        }
    }
}

template <int KMAX>
size_t persist_smem() {
    constexpr int D = 1 << KMAX;
    constexpr size_t a = PassSmem<(D < 4 ? 4 : D), kBlock>::bytes;
    constexpr size_t b = KMAX >= 3 ? blk::BlkSmem<(D >= 8 ? D : 8), kBlock>::bytes : 0;
    return a > b ? a : b;
}

template <int KMAX>
cudaError_t persist_prepare(int* blocks_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(persist_kernel<KMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)persist_smem<KMAX>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(class_pass_kernel<KMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)persist_smem<KMAX>());
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, persist_kernel<KMAX>, kBlock, persist_smem<KMAX>());
}

template <int KMAX>
cudaError_t persist_launch(const DevProblem& P, const PersistPlan& L, int grid, cudaStream_t s) {
    void* args[] = {const_cast<DevProblem*>(&P), const_cast<PersistPlan*>(&L)};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(persist_kernel<KMAX>), dim3(grid), dim3(kBlock), args,
                                       persist_smem<KMAX>(), s);
}

template <int D, int BLOCK>
cudaError_t set_pass_attr() {
    if constexpr (D == 32)
        return cudaFuncSetAttribute(region_pass_kernel32<BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)PassSmem<D, BLOCK>::bytes);
    else
        return cudaFuncSetAttribute(region_pass_kernel<D, BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)PassSmem<D, BLOCK>::bytes);
}

template <int D, int BLOCK>
cudaError_t launch_pass_DB(const DevProblem& P, const PassIO& io, const int32_t* cls, int32_t count, int k,
                           cudaStream_t s) {
    constexpr int G = BLOCK / D;
    const int64_t units = (int64_t)P.n_inst * count;
    const int64_t blocks = (units + G - 1) / G;
    if constexpr (D == 32)
        region_pass_kernel32<BLOCK><<<(unsigned)blocks, BLOCK, PassSmem<D, BLOCK>::bytes, s>>>(P, io, cls, count, k);
    else
        region_pass_kernel<D, BLOCK><<<(unsigned)blocks, BLOCK, PassSmem<D, BLOCK>::bytes, s>>>(P, io, cls, count, k);
    return cudaGetLastError();
}

template <int D>
cudaError_t launch_pass_D(const DevProblem& P, const PassIO& io, const int32_t* cls, int32_t count, int k,
                          cudaStream_t s, int block) {
    if (block == 64) return launch_pass_DB<D, 64>(P, io, cls, count, k, s);
    if (block == 256) return launch_pass_DB<D, 256>(P, io, cls, count, k, s);
    return launch_pass_DB<D, 128>(P, io, cls, count, k, s);
}

template <int D>
cudaError_t set_pass_attrs() {
    cudaError_t e;
    if ((e = set_pass_attr<D, 64>()) != cudaSuccess) return e;
    if ((e = set_pass_attr<D, 128>()) != cudaSuccess) return e;
    return set_pass_attr<D, 256>();
}

template <int D>
cudaError_t launch_cert_D(const DevProblem& P, const int32_t* cls, int32_t count, const float2* msg, cudaStream_t s) {
    constexpr int G = kBlock / D;
    const int64_t units = (int64_t)P.n_inst * count;
    const int64_t blocks = (units + G - 1) / G;
    certify_kernel<D><<<(unsigned)blocks, kBlock, CertSmem<D>::bytes, s>>>(P, cls, count, msg);
    return cudaGetLastError();
}

}  // namespace

cudaError_t prepare_kernels() {
    cudaError_t e;
    if ((e = set_pass_attrs<4>()) != cudaSuccess) return e;
    if ((e = set_pass_attrs<8>()) != cudaSuccess) return e;
    if ((e = set_pass_attrs<16>()) != cudaSuccess) return e;
    if ((e = set_pass_attrs<32>()) != cudaSuccess) return e;
    if ((e = prepare_blk_kernels()) != cudaSuccess) return e;
    return prepare_cta_kernels();
}

cudaError_t launch_region_pass(const DevProblem& P, const PassIO& io, int k, const int32_t* cls, int32_t count,
                               cudaStream_t s, int block) {
    if (count <= 0) return cudaSuccess;
    if (block > kShapeWarp16 && k == 4) return launch_region_pass_w16(P, io, cls, count, s, block - kShapeWarp16);
    if (block > kShapeBlocks && block < kShapeWarp16 && (k == 3 || k == 4))
        return launch_region_pass_blk(P, io, k, cls, count, s, block - kShapeBlocks);
    if (block > 0 && block != 64 && block != 256) block = 128;
    if (block < 0 && k != 2) block = 128;   // the one-thread-per-region layout exists for 4 x 4 only
    if (k == 1 && block < 0) block = 128;
    switch (k) {
        case 1: {
            const int64_t units = (int64_t)P.n_inst * count;
            region_pass_d2_kernel<<<(unsigned)((units + block - 1) / block), block, 0, s>>>(P, io, cls, count);
            return cudaGetLastError();
        }
        case 2: {
            if (block < 0) {
                const int tb = -block;
                const int64_t units = (int64_t)P.n_inst * count;
                const unsigned grid = (unsigned)((units + tb - 1) / tb);
                if (tb == 64) region_pass_t4_kernel<64><<<grid, 64, 0, s>>>(P, io, cls, count, k);
                else if (tb == 256) region_pass_t4_kernel<256><<<grid, 256, 0, s>>>(P, io, cls, count, k);
                else region_pass_t4_kernel<128><<<grid, 128, 0, s>>>(P, io, cls, count, k);
                return cudaGetLastError();
            }
            return launch_pass_D<4>(P, io, cls, count, k, s, block);
        }
        case 3: return launch_pass_D<8>(P, io, cls, count, k, s, block);
        case 4: return launch_pass_D<16>(P, io, cls, count, k, s, block);
        case 5: return launch_pass_D<32>(P, io, cls, count, k, s, block);
        case 6:
        case 7:
        case 8: return launch_region_pass_cta(P, io, k, cls, count, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_certify(const DevProblem& P, int k, const int32_t* cls, int32_t count, const float2* msg,
                           cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    switch (k) {
        case 1: {
            const int64_t units = (int64_t)P.n_inst * count;
            certify_d2_kernel<<<(unsigned)((units + kBlock - 1) / kBlock), kBlock, 0, s>>>(P, cls, count, msg);
            return cudaGetLastError();
        }
        case 2: return launch_cert_D<4>(P, cls, count, msg, s);
        case 3: return launch_cert_D<8>(P, cls, count, msg, s);
        case 4: return launch_cert_D<16>(P, cls, count, msg, s);
        case 5: return launch_cert_D<32>(P, cls, count, msg, s);
        case 6:
        case 7:
        case 8: return launch_certify_cta(P, k, cls, count, msg, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_update(const DevProblem& P, int par, int mode, cudaStream_t s) {
    const int64_t n = (int64_t)P.n_inst * (P.msg_elems >> 1);
    const int64_t blocks = (n + 255) / 256;
    update_kernel<<<(unsigned)(blocks > 0 ? blocks : 1), 256, 0, s>>>(P, par, mode);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const DevProblem& P, const PassIO& io, cudaStream_t s) {
    const int64_t n = (int64_t)P.n_inst * (P.msg_elems >> 1);
    if (n <= 0) return cudaSuccess;
    finalize_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P, io);
    return cudaGetLastError();
}

cudaError_t launch_halo_copy(const DevProblem& P, const int64_t* map, int64_t n_chunks, float2* buf, int unpack,
                             cudaStream_t s) {
    const int64_t n = (int64_t)P.n_inst * 2 * n_chunks;
    if (n <= 0) return cudaSuccess;
    halo_copy_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P, map, n_chunks, buf, unpack);
    return cudaGetLastError();
}

cudaError_t launch_advance(const DevProblem& P, int n, cudaStream_t s) {
    advance_kernel<<<1, 1, 0, s>>>(P.st, n);
    return cudaGetLastError();
}

int persistent_tile_regions(int k, int32_t blk_mask) {
    if (k == 4 && ((blk_mask >> 5) & 1)) return kBlock / 32;   // one warp per region
    return k == 1 ? kBlock : kBlock >> k;
}

cudaError_t persistent_prepare(int kmax, int* blocks_per_sm) {
    switch (kmax) {
        case 2: return persist_prepare<2>(blocks_per_sm);
        case 3: return persist_prepare<3>(blocks_per_sm);
        case 4: return persist_prepare<4>(blocks_per_sm);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_class_pass(const DevProblem& P, const PersistPlan& L, int kmax, const PassIO& io, cudaStream_t s) {
    const unsigned grid = (unsigned)L.tiles;
    switch (kmax) {
        case 2: class_pass_kernel<2><<<grid, kBlock, persist_smem<2>(), s>>>(P, L, io); break;
        case 3: class_pass_kernel<3><<<grid, kBlock, persist_smem<3>(), s>>>(P, L, io); break;
        case 4: class_pass_kernel<4><<<grid, kBlock, persist_smem<4>(), s>>>(P, L, io); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_persistent(const DevProblem& P, const PersistPlan& Lin, int kmax, int grid, cudaStream_t s,
                              bool unreleased) {
    PersistPlan L = Lin;
    // self-test: a barrier that expects one CTA more than the grid never opens
    L.expect = (unsigned)grid + (unreleased ? 1u : 0u);
    cudaError_t e = cudaMemsetAsync(L.bar, 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    switch (kmax) {
        case 2: return persist_launch<2>(P, L, grid, s);
        case 3: return persist_launch<3>(P, L, grid, s);
        case 4: return persist_launch<4>(P, L, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_reduce(const DevProblem& P, const double* vals, int track_best, cudaStream_t s) {
    reduce_kernel<<<P.n_inst, kReduce, 0, s>>>(P, vals, track_best);
    return cudaGetLastError();
}

cudaError_t launch_set_state(const DevProblem& P, int par, double theta, double t, int set_theta_t, double beta,
                             double inv_lhat, double alpha, double degen_tol, int variant, int step_rule,
                             int max_sweeps, int cert_sweeps, int cold, cudaStream_t s) {
    set_state_kernel<<<1, 1, 0, s>>>(P.st, par, theta, t, set_theta_t, beta, inv_lhat, alpha, degen_tol, variant,
                                     step_rule, max_sweeps, cert_sweeps, cold);
    return cudaGetLastError();
}

__global__ void round_terms_kernel(float2* __restrict__ h32, const double2* __restrict__ h64, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double2 v = h64[i];
        h32[i] = make_float2(__double2float_rn(v.x), __double2float_rn(v.y));
    }
}

cudaError_t launch_round_terms(float2* h32, const double2* h64, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 148 * 16);
    round_terms_kernel<<<(unsigned)blocks, 256, 0, s>>>(h32, h64, n);
    return cudaGetLastError();
}

cudaError_t launch_warm_identity(float2* warm, int64_t n_mats, int D, cudaStream_t s) {
    const int64_t pairs = n_mats * D * D / 2;
    if (pairs <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((pairs + 255) / 256, 148 * 16);
    warm_identity_kernel<<<(unsigned)blocks, 256, 0, s>>>(reinterpret_cast<float4*>(warm), pairs, D);
    return cudaGetLastError();
}

}  // namespace lrh
