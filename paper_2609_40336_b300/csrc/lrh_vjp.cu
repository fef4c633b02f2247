// Adjoint (reverse-mode derivative) of the smoothed region pass, sm_103a.
//
// Forward map at the evaluation point eta: (term matrices, multipliers) ->
//   Q_beta = sum_e F_beta(theta_e),  g_{e->f} = rho_f - Tr_{e\f} rho_e        (Sec. 4.1.2, 4.2)
// Given cotangents q_bar (per instance) and g_bar (message layout) this computes, per region,
//   rho_bar_e   = sum_{g in A(e)} g_bar_{g->e} - sum_{f in D(e)} 1 (x) g_bar_{e->f}
//                 (the same gather as theta with h = 0: adjoint of the partial trace),
//   theta_bar_e = V [ (V^dagger rho_bar V) o K + c diag(p) ] V^dagger,
//                 K_kl = (p_k - p_l) / (lambda_k - lambda_l), K_kk = -beta p_k,
//                 c = beta <rho_bar, rho> + q_bar          (dF_beta = <rho, dtheta>, and
//                 d rho = V [(V^dagger dtheta V) o K] V^dagger + beta <rho, dtheta> rho)
// with the eigenbasis recomputed (not stored), then
//   nu_bar_{e->f} = theta_bar_f - Tr_{e\f} theta_bar_e,   T_bar_t = Tr_{R\t} theta_bar_R.
// Layout: D lanes per region (lane-row Jacobi of lrh_device.cuh, 2 <= D <= 32); the four
// complex matrix products run from shared memory with one output row per lane.
#include "lrh_device.cuh"
#include "lrh_internal.cuh"

#include <cmath>
#include <cstdint>

namespace lrh {
namespace {

using namespace dev;
constexpr int kVB = 128;

template <int D>
struct VjpSmem {
    static constexpr int G = kVB / D;
    static constexpr int LD = D + 2;   // padded row stride (float2) of the staged matrices
    static constexpr size_t per_group = (D / 2 > 0 ? D / 2 : 1) * sizeof(Rot<float>) + 2 * D * sizeof(float) +
                                        2 * (size_t)D * LD * sizeof(float2);
    static constexpr size_t bytes = G * ((per_group + 15) / 16 * 16) + 16;
};

template <int D>
__global__ void __launch_bounds__(kVB) vjp_region_kernel(const DevProblem P, const int32_t* __restrict__ cls,
                                                         const int32_t count) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int G = kVB / D;
    const int g = threadIdx.x / D;
    const int s = threadIdx.x % D;
    unsigned char* base = smem_raw + g * ((VjpSmem<D>::per_group + 15) / 16 * 16);
    Rot<float>* prm = reinterpret_cast<Rot<float>*>(base);
    float* lam = reinterpret_cast<float*>(base + (D / 2 > 0 ? D / 2 : 1) * sizeof(Rot<float>));
    float* pp = lam + D;
    constexpr int LD = VjpSmem<D>::LD;
    float2* Vb = reinterpret_cast<float2*>(pp + D);
    float2* Yb = Vb + D * LD;

    const int64_t unit = (int64_t)blockIdx.x * G + g;
    const bool valid = unit < (int64_t)P.n_inst * count;
    const int inst = valid ? (int)(unit / count) : 0;
    const int r = valid ? cls[unit % count] : 0;
    const float th = (float)P.st->th3[P.st->t0 % 3];
    const float beta = (float)P.st->beta;

    float ar[D], ai[D], vr[D], vi[D];
    RegionInfo R;
    if (valid) {
        R = P.reg[r];
        assemble_row<D, float>(P, R, inst, s, P.nu, P.zeta, th, false, ar, ai);
    } else {
        R = RegionInfo{-1, -1, 0, 0, 0, 0, 0};
#pragma unroll
        for (int c = 0; c < D; ++c) { ar[c] = 0.f; ai[c] = 0.f; }
    }
#pragma unroll
    for (int c = 0; c < D; ++c) { vr[c] = (c == s) ? 1.f : 0.f; vi[c] = 0.f; }
    float norm2, off2;
    jacobi_lanes<D, float, true>(ar, ai, vr, vi, s, prm, P.st->max_sweeps, 1e-12f, norm2, off2);
    float e0, e1;
    pick_pair<D>(ar, s, e0, e1);
    const float lk = (s & 1) ? e1 : e0;
    const float lmin = group_min<D>(lk);
    const float ex = expf(-beta * (lk - lmin));
    const float Z = group_sum<D>(ex);
    lam[s] = lk;
    pp[s] = ex / Z;
    // rho_bar row s: gather of g_bar with h = 0
    if (valid) {
        RegionInfo R0 = R;
        R0.h_off = -1;
        assemble_row<D, float>(P, R0, inst, s, P.gbar, nullptr, 0.0f, false, ar, ai);
    }
#pragma unroll
    for (int c = 0; c < D; ++c) { Vb[s * LD + c] = make_float2(vr[c], vi[c]); Yb[s * LD + c] = make_float2(ar[c], ai[c]); }
    __syncwarp();
    // (1) Y = rho_bar V  (row s; own row of rho_bar from smem, rows of V broadcast)
    float yr[D], yi[D];
#pragma unroll
    for (int c = 0; c < D; ++c) { yr[c] = 0.f; yi[c] = 0.f; }
    for (int j = 0; j < D; ++j) {
        const float2 a = Yb[s * LD + j];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const float2 v = Vb[j * LD + c];
            yr[c] += a.x * v.x - a.y * v.y;
            yi[c] += a.x * v.y + a.y * v.x;
        }
    }
#pragma unroll
    for (int c = 0; c < D; ++c) Yb[s * LD + c] = make_float2(yr[c], yi[c]);   // own row only
    __syncwarp();
    // (2) M = V^dagger Y  (row k = s): M[k][c] = sum_i conj(V[i][k]) Y[i][c]
#pragma unroll
    for (int c = 0; c < D; ++c) { yr[c] = 0.f; yi[c] = 0.f; }
    for (int i = 0; i < D; ++i) {
        const float2 v = Vb[i * LD + s];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const float2 y = Yb[i * LD + c];
            yr[c] += v.x * y.x + v.y * y.y;
            yi[c] += v.x * y.y - v.y * y.x;
        }
    }
    // <rho_bar, rho> = sum_k p_k Re M_kk;   X = M o K + c diag(p)
    float mkk = 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c) mkk += (c == s) ? yr[c] : 0.f;
    const float inner = group_sum<D>(pp[s] * mkk);
    const float coef = beta * inner + (valid ? (float)P.qbar[inst] : 0.f);
    __syncwarp();
#pragma unroll
    for (int c = 0; c < D; ++c) {
        const float kv = kdd(lam[s], lam[c], pp[s], pp[c], beta);
        float xr = yr[c] * kv, xi = yi[c] * kv;
        if (c == s) xr += coef * pp[s];
        Yb[s * LD + c] = make_float2(xr, xi);
    }
    __syncwarp();
    // (3) Zr = V X  (row s; own row of V from smem, rows of X broadcast)
#pragma unroll
    for (int c = 0; c < D; ++c) { yr[c] = 0.f; yi[c] = 0.f; }
    for (int j = 0; j < D; ++j) {
        const float2 a = Vb[s * LD + j];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const float2 x = Yb[j * LD + c];
            yr[c] += a.x * x.x - a.y * x.y;
            yi[c] += a.x * x.y + a.y * x.x;
        }
    }
    __syncwarp();
    // (4) theta_bar = Zr V^dagger: theta_bar[s][j] = sum_c Zr[s][c] conj(V[j][c])
    for (int j = 0; j < D; ++j) {
        float tr_ = 0.f, ti_ = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const float2 v = Vb[j * LD + c];
            tr_ += yr[c] * v.x + yi[c] * v.y;
            ti_ += yi[c] * v.x - yr[c] * v.y;
        }
        Yb[s * LD + j] = make_float2(tr_, ti_);
    }
    __syncwarp();
    {
        float2 fix[D];
#pragma unroll
        for (int j = 0; j < D; ++j) { const float2 up = Yb[j * LD + s]; fix[j] = make_float2(up.x, -up.y); }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < D; ++j) {
            if (j < s) Yb[s * LD + j] = fix[j];
            if (j == s) Yb[s * LD + j].y = 0.f;
        }
    }
    __syncwarp();
    if (valid) {
        float2* dst = P.thb + (int64_t)inst * P.all_elems + R.all_off + (int64_t)s * D;
#pragma unroll
        for (int c = 0; c < D; ++c) dst[c] = Yb[s * LD + c];
        float2* trb = P.tr + (int64_t)inst * P.msg_elems;
        for (int q = R.child_begin; q < R.child_end; ++q) {
            const PairInfo pi = P.child_info[q];
            const int M = pi.mask, Mc = (D - 1) & ~M, kf = pi.kf, Df = 1 << kf, nrest = D >> kf;
            for (int idx = s; idx < Df * Df; idx += D) {
                const int ra = pdep_bits(idx >> kf, M), rb = pdep_bits(idx & (Df - 1), M);
                float sr = 0.f, si = 0.f;
                for (int c = 0; c < nrest; ++c) {
                    const int x = pdep_bits(c, Mc);
                    const float2 v = Yb[(ra | x) * LD + (rb | x)];
                    sr += v.x; si += v.y;
                }
                trb[pi.off + idx] = make_float2(sr, si);
            }
        }
    }
}

// nu_bar = theta_bar_f - Tr_{e\f} theta_bar_e  (one thread per complex entry)
__global__ void vjp_nubar_kernel(const DevProblem P, float2* __restrict__ nu_bar) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (int64_t)P.n_inst * P.msg_elems) return;
    const int inst = (int)(tid / P.msg_elems);
    const int64_t e = tid % P.msg_elems;
    const PairInfo pi = P.pair[P.chunk_pair[e >> 2]];
    const RegionInfo Rf = P.reg[pi.child];
    const float2 tf = P.thb[(int64_t)inst * P.all_elems + Rf.all_off + (e - pi.off)];
    const float2 tt = P.tr[(int64_t)inst * P.msg_elems + e];
    nu_bar[tid] = make_float2(tf.x - tt.x, tf.y - tt.y);
}

// T_bar_t = Tr_{R\t} theta_bar_R  (one thread per term-matrix entry)
__global__ void vjp_termbar_kernel(const DevProblem P, float2* __restrict__ term_bar) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per_inst = P.term_total;
    if (tid >= (int64_t)P.n_inst * per_inst) return;
    const int inst = (int)(tid / per_inst);
    const int64_t e = tid % per_inst;
    // term owning entry e: the largest t with out_off <= e
    int lo = 0, hi = P.n_terms - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.terms[mid].out_off <= e) lo = mid; else hi = mid - 1;
    }
    const TermInfo T = P.terms[lo];
    const RegionInfo R = P.reg[T.region];
    const int Dt = 1 << T.kt;
    const int DR = T.dr;
    const int64_t w = e - T.out_off;
    const int a = (int)(w / Dt), b = (int)(w % Dt);
    const int M = T.mask, Mc = (DR - 1) & ~M;
    const int ra = dev::pdep_bits(a, M), rb = dev::pdep_bits(b, M);
    const float2* th = P.thb + (int64_t)inst * P.all_elems + R.all_off;
    float sr = 0.f, si = 0.f;
    for (int c = 0; c < DR / Dt; ++c) {
        const int x = dev::pdep_bits(c, Mc);
        const float2 v = th[(int64_t)(ra | x) * DR + (rb | x)];
        sr += v.x; si += v.y;
    }
    term_bar[tid] = make_float2(sr, si);
}

template <int D>
cudaError_t vjp_D(const DevProblem& P, const int32_t* cls, int32_t count, cudaStream_t s) {
    constexpr int G = kVB / D;
    const int64_t units = (int64_t)P.n_inst * count;
    vjp_region_kernel<D><<<(unsigned)((units + G - 1) / G), kVB, VjpSmem<D>::bytes, s>>>(P, cls, count);
    return cudaGetLastError();
}

template <int D>
cudaError_t vjp_attr() {
    return cudaFuncSetAttribute(vjp_region_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)VjpSmem<D>::bytes);
}

}  // namespace

cudaError_t prepare_vjp_kernels() {
    cudaError_t e;
    if ((e = vjp_attr<2>()) != cudaSuccess) return e;
    if ((e = vjp_attr<4>()) != cudaSuccess) return e;
    if ((e = vjp_attr<8>()) != cudaSuccess) return e;
    if ((e = vjp_attr<16>()) != cudaSuccess) return e;
    return vjp_attr<32>();
}

cudaError_t launch_vjp_region(const DevProblem& P, int k, const int32_t* cls, int32_t count, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    switch (k) {
        case 1: return vjp_D<2>(P, cls, count, s);
        case 2: return vjp_D<4>(P, cls, count, s);
        case 3: return vjp_D<8>(P, cls, count, s);
        case 4: return vjp_D<16>(P, cls, count, s);
        case 5: return vjp_D<32>(P, cls, count, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_vjp_outputs(const DevProblem& P, float2* nu_bar, float2* term_bar, cudaStream_t s) {
    const int64_t nm = (int64_t)P.n_inst * P.msg_elems;
    if (nm > 0) vjp_nubar_kernel<<<(unsigned)((nm + 255) / 256), 256, 0, s>>>(P, nu_bar);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t nt = (int64_t)P.n_inst * P.term_total;
    if (nt > 0 && term_bar) vjp_termbar_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(P, term_bar);
    return cudaGetLastError();
}

}  // namespace lrh
