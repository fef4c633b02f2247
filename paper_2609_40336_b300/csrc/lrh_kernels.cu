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

#include <cfloat>
#include <cmath>
#include <cstdint>

namespace lrh {

namespace {

constexpr int kBlock = 128;
using namespace dev;

template <int D>
struct PassSmem {
    static constexpr int kGroups = kBlock / D;
    static constexpr size_t per_group = (D / 2) * sizeof(Rot<float>) + D * sizeof(float) + 2 * D * D * sizeof(float2);
    static constexpr size_t bytes = kGroups * per_group + 16;
};

// FP32 region pass for 4 <= D <= 32.
template <int D>
__global__ void __launch_bounds__(kBlock) region_pass_kernel(const DevProblem P, const int32_t* __restrict__ cls,
                                                             const int32_t count, const int par, const int k) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int G = kBlock / D;
    const int g = threadIdx.x / D;
    const int s = threadIdx.x % D;
    unsigned char* base = smem_raw + g * PassSmem<D>::per_group;
    Rot<float>* prm = reinterpret_cast<Rot<float>*>(base);
    float2* Wb = reinterpret_cast<float2*>(base + (D / 2) * sizeof(Rot<float>));
    float2* Rb = Wb + D * D;
    float* pw = reinterpret_cast<float*>(Rb + D * D);
    __shared__ unsigned long long blk_sweeps;
    if (threadIdx.x == 0) blk_sweeps = 0ull;

    const int64_t unit = (int64_t)blockIdx.x * G + g;
    const bool valid = unit < (int64_t)P.n_inst * count;
    const int inst = valid ? (int)(unit / count) : 0;
    const int r = valid ? cls[unit % count] : 0;
    const bool nest = P.st->variant == 1;
    const float th = nest ? (float)P.st->theta[par] : 0.0f;
    const int max_sweeps = P.st->max_sweeps;

    float ar[D], ai[D], vr[D], vi[D];
    RegionInfo R;
    if (valid) {
        R = P.reg[r];
        assemble_row<D, float>(P, R, inst, s, P.nu, nest ? P.zeta : nullptr, th, false, ar, ai);
    } else {
        R = RegionInfo{-1, -1, 0, 0, 0, 0};
#pragma unroll
        for (int c = 0; c < D; ++c) { ar[c] = 0.f; ai[c] = 0.f; }
    }
#pragma unroll
    for (int c = 0; c < D; ++c) { vr[c] = (c == s) ? 1.f : 0.f; vi[c] = 0.f; }

    float norm2;
    const int sweeps = jacobi_lanes<D, float, true>(ar, ai, vr, vi, s, prm, max_sweeps, 1e-12f, norm2);

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
        float4* wrow = reinterpret_cast<float4*>(Wb + s * D);
#pragma unroll
        for (int c = 0; c < D / 2; ++c) wrow[c] = make_float4(ar[2 * c], ai[2 * c], ar[2 * c + 1], ai[2 * c + 1]);
    }
    __syncwarp();
    for (int j = 0; j < D; ++j) {
        const float4* wj = reinterpret_cast<const float4*>(Wb + j * D);
        float accr = 0.f, acci = 0.f;
#pragma unroll
        for (int c = 0; c < D / 2; ++c) {
            const float4 x = wj[c];
            accr += ar[2 * c] * x.x + ai[2 * c] * x.y;
            acci += ai[2 * c] * x.x - ar[2 * c] * x.y;
            accr += ar[2 * c + 1] * x.z + ai[2 * c + 1] * x.w;
            acci += ai[2 * c + 1] * x.z - ar[2 * c + 1] * x.w;
        }
        Rb[s * D + j] = make_float2(accr, acci);
    }
    __syncwarp();
    // Make rho exactly Hermitian (the two triangles come from differently rounded sums):
    // row s keeps its upper part, takes the conjugate of the upper part for j < s, and a
    // real diagonal.  Exactly Hermitian states keep every message exactly Hermitian.
    {
        float2 fix[D];
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const float2 up = Rb[j * D + s];
            fix[j] = make_float2(up.x, -up.y);
        }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < D; ++j) {
            if (j < s) Rb[s * D + j] = fix[j];
            if (j == s) Rb[s * D + j].y = 0.f;
        }
    }
    __syncwarp();
    if (valid) {
        if (R.rho_off >= 0) {
            float4* dst = reinterpret_cast<float4*>(P.rho + (int64_t)inst * P.rho_elems + R.rho_off + (int64_t)s * D);
            const float4* srcr = reinterpret_cast<const float4*>(Rb + s * D);
#pragma unroll
            for (int c = 0; c < D / 2; ++c) dst[c] = srcr[c];
        }
        float2* trb = P.tr + (int64_t)inst * P.msg_elems;
        for (int q = R.child_begin; q < R.child_end; ++q) {
            const PairInfo pi = P.pair[P.child_pairs[q]];
            const int M = pi.mask;
            const int Mc = (D - 1) & ~M;
            const int kf = pi.kf;
            const int Df = 1 << kf;
            const int nrest = D >> kf;
            for (int idx = s; idx < Df * Df; idx += D) {
                const int ra = pdep_bits(idx >> kf, M);
                const int rb = pdep_bits(idx & (Df - 1), M);
                float accr = 0.f, acci = 0.f;
                for (int c = 0; c < nrest; ++c) {
                    const int x = pdep_bits(c, Mc);
                    const float2 v = Rb[(ra | x) * D + (rb | x)];
                    accr += v.x;
                    acci += v.y;
                }
                trb[pi.off + idx] = make_float2(accr, acci);
            }
        }
        if (s == 0) {
            P.val[(int64_t)inst * P.n_regions + r] = (double)F;
            if (!isfinite(F)) atomicOr(P.err, DEV_ERR_NUMERIC);
        }
    }
    // sweep accounting (regions x sweeps), one global atomic per block
    __syncthreads();
    if (valid && s == 0) atomicAdd(&blk_sweeps, (unsigned long long)sweeps);
    __syncthreads();
    if (threadIdx.x == 0 && blk_sweeps) atomicAdd(&P.sweeps[k], blk_sweeps);
}

// D = 2 closed form, one thread per region.  theta = m I + K, K = [[hh, b], [conj(b), -hh]],
// K^2 = r^2 I with r = sqrt(hh^2 + |b|^2): lambda = m -+ r,
// Gibbs state (1/2)(I - tanh(beta r) K / r), F_beta = m - r - log(1 + e^{-2 beta r}) / beta,
// ground projector (1/2)(I - K / r), or I/2 when 2r is within the degeneracy tolerance.
__global__ void __launch_bounds__(kBlock) region_pass_d2_kernel(const DevProblem P, const int32_t* __restrict__ cls,
                                                               const int32_t count, const int par) {
    const int64_t unit = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (unit >= (int64_t)P.n_inst * count) return;
    const int inst = (int)(unit / count);
    const int r = cls[unit % count];
    const bool nest = P.st->variant == 1;
    const float th = nest ? (float)P.st->theta[par] : 0.0f;
    const RegionInfo R = P.reg[r];
    float a = 0.f, d = 0.f, br = 0.f, bi = 0.f;
    if (R.h_off >= 0) {
        const float2* h = P.h32 + (int64_t)inst * P.h_elems + R.h_off;
        a = h[0].x; br = h[1].x; bi = h[1].y; d = h[3].x;
    }
    const int64_t mbase = (int64_t)inst * P.msg_elems;
    const float om = 1.0f - th;
    for (int q = R.parent_begin; q < R.parent_end; ++q) {
        const PairInfo pi = P.pair[P.parent_pairs[q]];
        const float4* nb = reinterpret_cast<const float4*>(P.nu + mbase + pi.off);
        float4 m0 = nb[0], m1 = nb[1];
        if (nest) {
            const float4* zb = reinterpret_cast<const float4*>(P.zeta + mbase + pi.off);
            const float4 z0 = zb[0], z1 = zb[1];
            m0.x = om * m0.x + th * z0.x; m0.z = om * m0.z + th * z0.z; m0.w = om * m0.w + th * z0.w;
            m1.z = om * m1.z + th * z1.z;
        }
        a += m0.x; br += m0.z; bi += m0.w; d += m1.z;
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
        float4* dst = reinterpret_cast<float4*>(P.rho + (int64_t)inst * P.rho_elems + R.rho_off);
        dst[0] = make_float4(0.5f * (1.f - kap * hh), 0.f, -0.5f * kap * br, -0.5f * kap * bi);
        dst[1] = make_float4(-0.5f * kap * br, 0.5f * kap * bi, 0.5f * (1.f + kap * hh), 0.f);
    }
    P.val[(int64_t)inst * P.n_regions + r] = (double)F;
    if (!isfinite(F)) atomicOr(P.err, DEV_ERR_NUMERIC);
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
    double norm2;
    jacobi_lanes<D, double, false>(ar, ai, vr, vi, s, prm, 40, 1e-28, norm2);
    double e0, e1;
    pick_pair<D>(ar, s, e0, e1);
    const double lam = (s & 1) ? e1 : e0;
    const double lmin = group_min<D>(lam);
    if (valid && s == 0) {
        P.val64[(int64_t)inst * P.n_regions + r] = lmin;
        if (!isfinite(lmin)) atomicOr(P.err, DEV_ERR_NUMERIC);
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
        const PairInfo pi = P.pair[P.parent_pairs[q]];
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
__global__ void update_kernel(const DevProblem P, const int par, const int mode) {
    const int64_t halfm = P.msg_elems >> 1;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double thd = P.st->theta[par];
    const double td = P.st->t[par];
    if (tid == 0 && mode == UPD_STEP) {
        // scalars of the next iteration (other parity slot)
        P.st->theta[par ^ 1] = (sqrt(thd * thd * thd * thd + 4.0 * thd * thd) - thd * thd) * 0.5;
        P.st->t[par ^ 1] = td + 1.0;
    }
    if (tid >= (int64_t)P.n_inst * halfm) return;
    const int inst = (int)(tid / halfm);
    const int64_t e = (tid % halfm) * 2;
    const int p = P.chunk_pair[e >> 2];
    const PairInfo pi = P.pair[p];
    const RegionInfo Rf = P.reg[pi.child];
    const int64_t mi = (int64_t)inst * P.msg_elems + e;
    const float4 rf = *reinterpret_cast<const float4*>(P.rho + (int64_t)inst * P.rho_elems + Rf.rho_off + (e - pi.off));
    const float4 tv = *reinterpret_cast<const float4*>(P.tr + mi);
    const float4 gv = make_float4(rf.x - tv.x, rf.y - tv.y, rf.z - tv.z, rf.w - tv.w);
    if (mode == UPD_GRAD_ONLY) {
        *reinterpret_cast<float4*>(P.grad + mi) = gv;
        return;
    }
    float4 nv = *reinterpret_cast<const float4*>(P.nu + mi);
    if (P.st->variant == 1) {
        const float th = (float)thd;
        const float kz = (float)(P.st->inv_lhat / thd);
        float4 z = *reinterpret_cast<const float4*>(P.zeta + mi);
        z.x = fmaf(kz, gv.x, z.x); z.y = fmaf(kz, gv.y, z.y); z.z = fmaf(kz, gv.z, z.z); z.w = fmaf(kz, gv.w, z.w);
        const float om = 1.0f - th;
        nv.x = fmaf(th, z.x, om * nv.x); nv.y = fmaf(th, z.y, om * nv.y);
        nv.z = fmaf(th, z.z, om * nv.z); nv.w = fmaf(th, z.w, om * nv.w);
        *reinterpret_cast<float4*>(P.zeta + mi) = z;
    } else {
        if (P.best_flag[inst]) *reinterpret_cast<float4*>(P.nu_best + mi) = nv;
        const double a0 = P.st->alpha;
        const float alpha = (float)(P.st->step_rule == 1 ? a0 / sqrt(td + 1.0) : a0);
        nv.x = fmaf(alpha, gv.x, nv.x); nv.y = fmaf(alpha, gv.y, nv.y);
        nv.z = fmaf(alpha, gv.z, nv.z); nv.w = fmaf(alpha, gv.w, nv.w);
    }
    if (!(isfinite(nv.x) && isfinite(nv.y) && isfinite(nv.z) && isfinite(nv.w))) atomicOr(P.err, DEV_ERR_NUMERIC);
    *reinterpret_cast<float4*>(P.nu + mi) = nv;
}

// Deterministic per-instance FP64 sum of per-region values (fixed strided partial sums and a
// fixed tree), with optional Alg. 1 best-so-far tracking.
constexpr int kReduce = 256;
__global__ void __launch_bounds__(kReduce) reduce_kernel(const DevProblem P, const double* __restrict__ vals,
                                                        const int track_best) {
    __shared__ double sh[kReduce];
    const int inst = blockIdx.x;
    const double* v = vals + (int64_t)inst * P.n_regions;
    double acc = 0.0;
    for (int i = threadIdx.x; i < P.n_regions; i += kReduce) acc += v[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kReduce / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
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

__global__ void set_state_kernel(IterState* st, int par, double theta, double t, int set_theta_t, double beta,
                                 double inv_lhat, double alpha, double degen_tol, int variant, int step_rule,
                                 int max_sweeps) {
    if (set_theta_t) { st->theta[par] = theta; st->t[par] = t; }
    st->beta = beta;
    st->inv_lhat = inv_lhat;
    st->alpha = alpha;
    st->degen_tol = degen_tol;
    st->variant = variant;
    st->step_rule = step_rule;
    st->max_sweeps = max_sweeps;
}

template <int D>
cudaError_t set_pass_attr() {
    return cudaFuncSetAttribute(region_pass_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)PassSmem<D>::bytes);
}

template <int D>
cudaError_t launch_pass_D(const DevProblem& P, const int32_t* cls, int32_t count, int par, int k, cudaStream_t s) {
    const size_t smem = PassSmem<D>::bytes;
    constexpr int G = kBlock / D;
    const int64_t units = (int64_t)P.n_inst * count;
    const int64_t blocks = (units + G - 1) / G;
    region_pass_kernel<D><<<(unsigned)blocks, kBlock, smem, s>>>(P, cls, count, par, k);
    return cudaGetLastError();
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
    if ((e = set_pass_attr<4>()) != cudaSuccess) return e;
    if ((e = set_pass_attr<8>()) != cudaSuccess) return e;
    if ((e = set_pass_attr<16>()) != cudaSuccess) return e;
    if ((e = set_pass_attr<32>()) != cudaSuccess) return e;
    return prepare_cta_kernels();
}

cudaError_t launch_region_pass(const DevProblem& P, int k, const int32_t* cls, int32_t count, int par,
                               cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    switch (k) {
        case 1: {
            const int64_t units = (int64_t)P.n_inst * count;
            region_pass_d2_kernel<<<(unsigned)((units + kBlock - 1) / kBlock), kBlock, 0, s>>>(P, cls, count, par);
            return cudaGetLastError();
        }
        case 2: return launch_pass_D<4>(P, cls, count, par, k, s);
        case 3: return launch_pass_D<8>(P, cls, count, par, k, s);
        case 4: return launch_pass_D<16>(P, cls, count, par, k, s);
        case 5: return launch_pass_D<32>(P, cls, count, par, k, s);
        case 6:
        case 7: return launch_region_pass_cta(P, k, cls, count, par, s);
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
        case 7: return launch_certify_cta(P, k, cls, count, msg, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_update(const DevProblem& P, int par, int mode, cudaStream_t s) {
    const int64_t n = (int64_t)P.n_inst * (P.msg_elems >> 1);
    const int64_t blocks = (n + 255) / 256;
    update_kernel<<<(unsigned)(blocks > 0 ? blocks : 1), 256, 0, s>>>(P, par, mode);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const DevProblem& P, const double* vals, int track_best, cudaStream_t s) {
    reduce_kernel<<<P.n_inst, kReduce, 0, s>>>(P, vals, track_best);
    return cudaGetLastError();
}

cudaError_t launch_set_state(const DevProblem& P, int par, double theta, double t, int set_theta_t, double beta,
                             double inv_lhat, double alpha, double degen_tol, int variant, int step_rule,
                             int max_sweeps, cudaStream_t s) {
    set_state_kernel<<<1, 1, 0, s>>>(P.st, par, theta, t, set_theta_t, beta, inv_lhat, alpha, degen_tol, variant,
                                     step_rule, max_sweeps);
    return cudaGetLastError();
}

}  // namespace lrh
