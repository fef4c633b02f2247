// Device helpers of the lane-row complex Jacobi eigensolver (4 <= D <= 32) shared by the
// kernel files.  See lrh_kernels.cu for the layout.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "lrh_internal.cuh"

namespace lrh {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;

// Source slot of the round-robin tournament: after a round, slot s receives the content of
// slot rr_src(s).  Slot 0 is fixed, the other D-1 slots form one cycle, so D-1 rounds visit
// every unordered pair exactly once and restore the natural order.
__host__ __device__ constexpr int rr_src(int s, int D) {
    return D == 2 ? s : s == 0 ? 0 : (s == 2 ? 1 : ((s & 1) == 0 ? s - 2 : (s == D - 1 ? D - 2 : s + 2)));
}

__device__ __forceinline__ int pext_bits(int x, int m) {
    int r = 0, k = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        if ((m >> b) & 1) { r |= ((x >> b) & 1) << k; ++k; }
    }
    return r;
}

__device__ __forceinline__ int pdep_bits(int x, int m) {
    int r = 0, k = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        if ((m >> b) & 1) { r |= ((x >> k) & 1) << b; ++k; }
    }
    return r;
}

template <int W, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o, W);
    return v;
}

template <int W, typename T>
__device__ __forceinline__ T group_min(T v) {
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) {
        T u = __shfl_xor_sync(kFull, v, o, W);
        v = u < v ? u : v;
    }
    return v;
}

template <typename T> struct alignas(4 * sizeof(T)) Rot { T c, wr, wi, pad; };

__device__ __forceinline__ float my_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double my_sqrt(double x) { return sqrt(x); }

// Jacobi rotation of the Hermitian 2x2 block [[app, b], [conj(b), aqq]]:
// J = [[c, -w], [conj(w), c]] with w = sigma b, sigma real, makes (J^H A J)_pq = 0.
// With h = aqq - app and r = sqrt(h^2 + 4|b|^2): t = -sgn(h) 2|b| / (|h| + r),
// c = 1 / sqrt(1 + t^2), sigma = -sgn(h) 2 c / (|h| + r)  (no division by |b|).
template <typename T>
__device__ __forceinline__ void rot_params(T app, T aqq, T br, T bi, T& c, T& wr, T& wi) {
    const T h = aqq - app;
    const T b2 = br * br + bi * bi;
    const T r = my_sqrt(h * h + T(4) * b2);
    const T den = fabs(h) + r;
    const T sg = h >= T(0) ? T(1) : T(-1);
    T t = T(0), sig = T(0);
    if (den > T(0)) t = -sg * T(2) * my_sqrt(b2) / den;
    c = T(1) / my_sqrt(T(1) + t * t);
    if (den > T(0)) sig = -sg * T(2) * c / den;
    wr = sig * br;
    wi = sig * bi;
}

// x[s & ~1] and x[s | 1] of a register row, by a select tree on the bits of s above bit 0.
// Template recursion keeps every register index a compile-time constant.
template <int HALF, int D, typename T>
struct PickLevel {
    static __device__ __forceinline__ void run(T (&t)[D], int s) {
        const bool hi = (s & HALF) != 0;
#pragma unroll
        for (int j = 0; j < HALF; ++j) t[j] = hi ? t[j + HALF] : t[j];
        PickLevel<HALF / 2, D, T>::run(t, s);
    }
};
template <int D, typename T>
struct PickLevel<1, D, T> {
    static __device__ __forceinline__ void run(T (&)[D], int) {}
};

template <int D, typename T>
__device__ __forceinline__ void pick_pair(const T (&x)[D], int s, T& x0, T& x1) {
    T t[D];
#pragma unroll
    for (int j = 0; j < D; ++j) t[j] = x[j];
    PickLevel<D / 2, D, T>::run(t, s);
    x0 = t[0];
    x1 = t[1];
}

// Column rotation of slots (p, q) = (2k, 2k+1): x_p' = c x_p + conj(w) x_q, x_q' = -w x_p + c x_q.
template <typename T>
__device__ __forceinline__ void mix_cols(T& pr, T& pi, T& qr, T& qi, T c, T wr, T wi) {
    const T npr = c * pr + (wr * qr + wi * qi);
    const T npi = c * pi + (wr * qi - wi * qr);
    const T nqr = c * qr - (wr * pr - wi * pi);
    const T nqi = c * qi - (wr * pi + wi * pr);
    pr = npr; pi = npi; qr = nqr; qi = nqi;
}

// ------------------------------------------------------------------ 2x2-block Jacobi helpers
template <typename T> struct Cplx;
template <> struct Cplx<float> { using t = float2; };
template <> struct Cplx<double> { using t = double2; };

template <typename T> struct alignas(4 * sizeof(T)) RotC { T c, wr, wi, pad; };

// Rotation J = [[c, -w], [conj(w), c]], w = sigma a_pq, of pair (p, q) from a_pp, a_qq, a_pq
// (h = a_qq - a_pp, r = sqrt(h^2 + 4|a_pq|^2), t = -sgn(h) 2|a_pq| / (|h| + r), c = 1 / sqrt(1 + t^2),
// sigma = -sgn(h) 2 c / (|h| + r)), and the diagonal after it, a_pp + t |a_pq| and a_qq - t |a_pq|.
template <typename T>
__device__ __forceinline__ void rot_params_d(T app, T aqq, T br, T bi, RotC<T>& R, typename Cplx<T>::t& dnew) {
    const T h = aqq - app;
    const T b2 = br * br + bi * bi;
    const T r = my_sqrt(h * h + T(4) * b2);
    const T den = fabs(h) + r;
    const T sg = h >= T(0) ? T(1) : T(-1);
    const T bn = my_sqrt(b2);
    T t = T(0), sig = T(0);
    if (den > T(0)) t = -sg * T(2) * bn / den;
    const T c = T(1) / my_sqrt(T(1) + t * t);
    if (den > T(0)) sig = -sg * T(2) * c / den;
    R.c = c;
    R.wr = sig * br;
    R.wi = sig * bi;
    R.pad = T(0);
    dnew.x = app + t * bn;
    dnew.y = aqq - t * bn;
}

// B' = J_k^H B J_l on a 2x2 block, J = [[c, -w], [conj(w), c]].
template <typename T, typename C2>
__device__ __forceinline__ void two_sided(C2& b00, C2& b01, C2& b10, C2& b11, const RotC<T>& K, const RotC<T>& Lr) {
    // C = B J_l : x_p' = c x_p + conj(w) x_q ; x_q' = -w x_p + c x_q   (per row)
    auto colmix = [&](C2& xp, C2& xq) {
        const T pr = Lr.c * xp.x + (Lr.wr * xq.x + Lr.wi * xq.y);
        const T pi = Lr.c * xp.y + (Lr.wr * xq.y - Lr.wi * xq.x);
        const T qr = Lr.c * xq.x - (Lr.wr * xp.x - Lr.wi * xp.y);
        const T qi = Lr.c * xq.y - (Lr.wr * xp.y + Lr.wi * xp.x);
        xp.x = pr; xp.y = pi; xq.x = qr; xq.y = qi;
    };
    colmix(b00, b01);
    colmix(b10, b11);
    // J_k^H C : y_p' = c y_p + w y_q ; y_q' = -conj(w) y_p + c y_q   (per column)
    auto rowmix = [&](C2& yp, C2& yq) {
        const T pr = K.c * yp.x + (K.wr * yq.x - K.wi * yq.y);
        const T pi = K.c * yp.y + (K.wr * yq.y + K.wi * yq.x);
        const T qr = K.c * yq.x - (K.wr * yp.x + K.wi * yp.y);
        const T qi = K.c * yq.y - (K.wr * yp.y - K.wi * yp.x);
        yp.x = pr; yp.y = pi; yq.x = qr; yq.y = qi;
    };
    rowmix(b00, b10);
    rowmix(b01, b11);
}

// Cyclic complex Jacobi on the D x D Hermitian matrix held by a group of D lanes (row per
// lane).  Returns the sweeps run (uniform over the warp).  On return the slots are in natural
// order: lane s holds lambda_s on its diagonal entry and, if WANT_V, row s of V whose column c
// is the eigenvector of lambda_c.  `norm2` receives ||theta||_F^2 and `off2` the squared
// Frobenius norm of the off-diagonal part left at exit (at most tol2 * norm2 unless the sweep
// cap stopped the iteration first).
template <int D, typename T, bool WANT_V>
__device__ __forceinline__ int jacobi_lanes(T (&ar)[D], T (&ai)[D], T (&vr)[D], T (&vi)[D], const int s,
                                            Rot<T>* prm, const int max_sweeps, const T tol2, T& norm2, T& off2) {
    T n2 = T(0);
#pragma unroll
    for (int c = 0; c < D; ++c) n2 += ar[c] * ar[c] + ai[c] * ai[c];
    n2 = group_sum<D>(n2);
    norm2 = n2;
    const T thresh = tol2 * n2;
    // Each group (region) stops at its own test; while other groups of the warp still sweep, a
    // stopped group runs identity rotations (c = 1, w = 0: every value is kept exactly and only
    // the tournament permutation moves it, which whole sweeps undo), so a region's result does
    // not depend on the regions that share its warp.
    int sweeps = 0;
    bool active = true;
    for (;;) {
        T off = T(0);
#pragma unroll
        for (int c = 0; c < D; ++c) off += (c == s) ? T(0) : (ar[c] * ar[c] + ai[c] * ai[c]);
        off = group_sum<D>(off);
        if (active) {
            off2 = off;
            active = !((off <= thresh) || (sweeps >= max_sweeps));
        }
        if (!__any_sync(kFull, active)) break;
        if (active) ++sweeps;
        // One round of the tournament: pair parameters from (xr, xi), column rotations of
        // (xr, xi) and of V (ur, ui) in place, the row rotation with the tournament permutation
        // into (yr, yi) and V's column permutation into (wr_, wi_).  Rounds alternate between
        // the two register arrays of each matrix (no copies).
        auto round = [&](T (&xr)[D], T (&xi)[D], T (&yr)[D], T (&yi)[D], T (&ur)[D], T (&ui)[D], T (&wr_)[D], T (&wi_)[D]) {
            // (1) parameters of pair k = s >> 1 (both lanes of the pair compute them from the
            //     same shuffled values, so they agree bit for bit)
            T e0r, e1r, e0i, e1i;
            pick_pair<D>(xr, s, e0r, e1r);
            pick_pair<D>(xi, s, e0i, e1i);
            const bool odd = (s & 1) != 0;
            const T mydiag = odd ? e1r : e0r;
            const T offr = odd ? e0r : e1r;
            const T offi = odd ? e0i : e1i;
            const T pdiag = __shfl_xor_sync(kFull, mydiag, 1, D);
            const T br = __shfl_sync(kFull, offr, s & ~1, D);
            const T bi = __shfl_sync(kFull, offi, s & ~1, D);
            const T app = odd ? pdiag : mydiag;
            const T aqq = odd ? mydiag : pdiag;
            T c, wr, wi;
            rot_params(app, aqq, br, bi, c, wr, wi);
            if (!active) { c = T(1); wr = T(0); wi = T(0); }
            if (!odd) prm[s >> 1] = Rot<T>{c, wr, wi, T(0)};
            __syncwarp();
            // (2) column rotations of A and V (all pairs)
#pragma unroll
            for (int k = 0; k < D / 2; ++k) {
                const Rot<T> P = prm[k];
                mix_cols(xr[2 * k], xi[2 * k], xr[2 * k + 1], xi[2 * k + 1], P.c, P.wr, P.wi);
                if (WANT_V) mix_cols(ur[2 * k], ui[2 * k], ur[2 * k + 1], ui[2 * k + 1], P.c, P.wr, P.wi);
            }
            // (3) row rotation fused with the tournament permutation of rows and columns:
            //     new A[s][c] = (J^H A)[o][rr_src(c)] with o = rr_src(s); for an odd source row
            //     the sign of the rotation's second term is folded into its coefficients
            const int o = rr_src(s, D);
            const Rot<T> Q = prm[o >> 1];
            const bool oodd = (o & 1) != 0;
            const T qwr = oodd ? -Q.wr : Q.wr;
            const T qwi = Q.wi;
#pragma unroll
            for (int cc = 0; cc < D; ++cc) {
                const int sc = rr_src(cc, D);
                const T r1r = __shfl_sync(kFull, xr[sc], o, D);
                const T r1i = __shfl_sync(kFull, xi[sc], o, D);
                const T r2r = __shfl_sync(kFull, xr[sc], o ^ 1, D);
                const T r2i = __shfl_sync(kFull, xi[sc], o ^ 1, D);
                yr[cc] = Q.c * r1r + (qwr * r2r - qwi * r2i);
                yi[cc] = Q.c * r1i + (qwr * r2i + qwi * r2r);
            }
            if (WANT_V) {
#pragma unroll
                for (int cc = 0; cc < D; ++cc) { wr_[cc] = ur[rr_src(cc, D)]; wi_[cc] = ui[rr_src(cc, D)]; }
            }
            __syncwarp();
        };
        T br_[D], bi_[D], ubr[D], ubi[D];
#pragma unroll 1
        for (int r = 0; r + 1 < D - 1; r += 2) {
            round(ar, ai, br_, bi_, vr, vi, ubr, ubi);
            round(br_, bi_, ar, ai, ubr, ubi, vr, vi);
        }
        // D - 1 rounds per sweep is odd: the last one lands in (br_, bi_) and (ubr, ubi)
        round(ar, ai, br_, bi_, vr, vi, ubr, ubi);
#pragma unroll
        for (int cc = 0; cc < D; ++cc) { ar[cc] = br_[cc]; ai[cc] = bi_[cc]; }
        if (WANT_V) {
#pragma unroll
            for (int cc = 0; cc < D; ++cc) { vr[cc] = ubr[cc]; vi[cc] = ubi[cc]; }
        }
    }
    return sweeps;
}

// Gather row s of theta_e = h_e - sum_children 1 (x) m_{e->f} + sum_parents m_{g->e}, with the
// message m = (1 - th) nu + th zeta (th = 0 for nu alone).  Source element type S, target T.
template <int D, typename T>
__device__ __forceinline__ void assemble_row(const DevProblem& P, const RegionInfo& R, int inst, int s,
                                             const float2* __restrict__ nu, const float2* __restrict__ zeta,
                                             float th, bool use_h64, T (&ar)[D], T (&ai)[D]) {
    if (R.h_off >= 0) {
        if (use_h64) {
            const double2* hrow = P.h64 + (int64_t)inst * P.h_elems + R.h_off + (int64_t)s * D;
#pragma unroll
            for (int c = 0; c < D; ++c) { const double2 v = hrow[c]; ar[c] = T(v.x); ai[c] = T(v.y); }
        } else {
            const float4* hrow = reinterpret_cast<const float4*>(P.h32 + (int64_t)inst * P.h_elems + R.h_off + (int64_t)s * D);
#pragma unroll
            for (int c = 0; c < D / 2; ++c) {
                const float4 v = hrow[c];
                ar[2 * c] = T(v.x); ai[2 * c] = T(v.y); ar[2 * c + 1] = T(v.z); ai[2 * c + 1] = T(v.w);
            }
        }
    } else {
#pragma unroll
        for (int c = 0; c < D; ++c) { ar[c] = T(0); ai[c] = T(0); }
    }
    const int64_t mbase = (int64_t)inst * P.msg_elems;
    const float om = 1.0f - th;
    for (int q = R.child_begin; q < R.child_end; ++q) {
        const PairInfo pi = P.child_info[q];
        const int M = pi.mask;
        const int Df = 1 << pi.kf;
        const int a = pext_bits(s, M);
        const int rest = s & ~M;
        const float2* nb = nu + mbase + pi.off + (int64_t)a * Df;
        const float2* zb = zeta ? zeta + mbase + pi.off + (int64_t)a * Df : nullptr;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            if ((c & ~M) == rest) {
                const int b = pext_bits(c, M);
                float2 m = nb[b];
                if (zb) { const float2 z = zb[b]; m.x = om * m.x + th * z.x; m.y = om * m.y + th * z.y; }
                ar[c] -= T(m.x);
                ai[c] -= T(m.y);
            }
        }
    }
    for (int q = R.parent_begin; q < R.parent_end; ++q) {
        const PairInfo pi = P.parent_info[q];
        const float4* nb = reinterpret_cast<const float4*>(nu + mbase + pi.off + (int64_t)s * D);
        const float4* zb = zeta ? reinterpret_cast<const float4*>(zeta + mbase + pi.off + (int64_t)s * D) : nullptr;
#pragma unroll
        for (int c = 0; c < D / 2; ++c) {
            float4 m = nb[c];
            if (zb) {
                const float4 z = zb[c];
                m.x = om * m.x + th * z.x; m.y = om * m.y + th * z.y;
                m.z = om * m.z + th * z.z; m.w = om * m.w + th * z.w;
            }
            ar[2 * c] += T(m.x); ai[2 * c] += T(m.y); ar[2 * c + 1] += T(m.z); ai[2 * c + 1] += T(m.w);
        }
    }
}

// K_kl of the eigendecomposition's adjoint for lambda_k, lambda_l with Gibbs weights p_k, p_l:
// the divided difference (p_k - p_l) / (lambda_k - lambda_l) of the normalised e^{-beta x},
// evaluated stably as p_lo expm1(-beta |d|) / |d| (p_lo = weight of the smaller eigenvalue),
// with the limit -beta p at coinciding eigenvalues.
__device__ __forceinline__ float kdd(float lk, float ll, float pk, float pl, float beta) {
    const float d = fabsf(lk - ll);
    const float plo = lk <= ll ? pk : pl;
    if (d * beta < 1e-6f) return -beta * plo;
    return plo * expm1f(-beta * d) / d;
}

// ------------------------------------------------------------------ fused Alg. 2 passes
struct Thetas {
    float cur;    // theta_t of this pass (extrapolation eta = (1 - theta_t) nu + theta_t zeta)
    float prev;   // theta_{t-1} of the pending update
    float kz;     // 1 / (theta_{t-1} L_hat)
};

__device__ __forceinline__ Thetas pass_thetas(const DevProblem& P, const PassIO& io) {
    Thetas T{0.f, 0.f, 0.f};
    if (!io.zeta_in) return T;
    const long long t = P.st->t0 + io.rel;
    T.cur = (float)P.st->th3[t % 3];
    if (io.pending) {
        const double tp = P.st->th3[(t + 2) % 3];
        T.prev = (float)tp;
        T.kz = (float)(P.st->inv_lhat / tp);
    }
    return T;
}

// The launch marked `writer` of a pass stores theta_{t+1} = (sqrt(theta^4 + 4 theta^2) - theta^2)/2
// (Alg. 2) in slot (t + 1) mod 3; the pass itself reads slots t and t - 1 only.
__device__ __forceinline__ void advance_theta(const DevProblem& P, const PassIO& io) {
    if (!io.zeta_in) return;
    const long long t = P.st->t0 + io.rel;
    const double th = P.st->th3[t % 3];
    P.st->th3[(t + 1) % 3] = (sqrt(th * th * th * th + 4.0 * th * th) - th * th) * 0.5;
}

// Alg. 2 update of one message entry: zeta += kz g, nu = (1 - theta) nu + theta zeta.
__device__ __forceinline__ void nesterov_update(float2& n, float2& z, float gx, float gy, float th, float kz) {
    z.x = fmaf(kz, gx, z.x);
    z.y = fmaf(kz, gy, z.y);
    const float om = 1.0f - th;
    n.x = fmaf(th, z.x, om * n.x);
    n.y = fmaf(th, z.y, om * n.y);
}

__device__ __forceinline__ float2 extrapolate(float2 n, float2 z, float th) {
    const float om = 1.0f - th;
    return make_float2(fmaf(th, z.x, om * n.x), fmaf(th, z.y, om * n.y));
}

// Message entry seen by a pass: nu (Alg. 1), or eta after applying the pending update
// (Alg. 2).  `mi` indexes the message arrays, `ri` the child's state of the previous pass.
// The owner (the pair's child region) stores the updated nu, zeta; n_out / z_out return them.
__device__ __forceinline__ float2 pass_entry(const PassIO& io, const Thetas& T, int64_t mi, int64_t ri, bool owner,
                                             float2* n_out = nullptr, float2* z_out = nullptr) {
    float2 n = io.nu_in[mi];
    if (!io.zeta_in) return n;
    float2 z = io.zeta_in[mi];
    if (io.pending) {
        const float2 r = io.rho_in[ri], t = io.tr_in[mi];
        nesterov_update(n, z, r.x - t.x, r.y - t.y, T.prev, T.kz);
        if (owner) { io.nu_out[mi] = n; io.zeta_out[mi] = z; }
    }
    if (n_out) *n_out = n;
    if (z_out) *z_out = z;
    return extrapolate(n, z, T.cur);
}

// Two consecutive entries (mi, ri even: 16-byte aligned) with float4 loads and stores; the same
// per-entry arithmetic as pass_entry.
__device__ __forceinline__ float4 pass_entry2(const PassIO& io, const Thetas& T, int64_t mi, int64_t ri, bool owner) {
    float4 n = *reinterpret_cast<const float4*>(io.nu_in + mi);
    if (!io.zeta_in) return n;
    float4 z = *reinterpret_cast<const float4*>(io.zeta_in + mi);
    if (io.pending) {
        const float4 r = *reinterpret_cast<const float4*>(io.rho_in + ri);
        const float4 t = *reinterpret_cast<const float4*>(io.tr_in + mi);
        float2 n0 = make_float2(n.x, n.y), n1 = make_float2(n.z, n.w);
        float2 z0 = make_float2(z.x, z.y), z1 = make_float2(z.z, z.w);
        nesterov_update(n0, z0, r.x - t.x, r.y - t.y, T.prev, T.kz);
        nesterov_update(n1, z1, r.z - t.z, r.w - t.w, T.prev, T.kz);
        n = make_float4(n0.x, n0.y, n1.x, n1.y);
        z = make_float4(z0.x, z0.y, z1.x, z1.y);
        if (owner) {
            *reinterpret_cast<float4*>(io.nu_out + mi) = n;
            *reinterpret_cast<float4*>(io.zeta_out + mi) = z;
        }
    }
    const float2 e0 = extrapolate(make_float2(n.x, n.y), make_float2(z.x, z.y), T.cur);
    const float2 e1 = extrapolate(make_float2(n.z, n.w), make_float2(z.z, z.w), T.cur);
    return make_float4(e0.x, e0.y, e1.x, e1.y);
}

// Row s of theta_e for an FP32 pass: h_e - sum_children 1 (x) m + sum_parents m with the
// message entries of pass_entry.
template <int D>
__device__ __forceinline__ void assemble_row_io(const DevProblem& P, const RegionInfo& R, int inst, int s,
                                                const PassIO& io, const Thetas& T, float (&ar)[D], float (&ai)[D]) {
    if (R.h_off >= 0) {
        const float4* hrow = reinterpret_cast<const float4*>(P.h32 + (int64_t)inst * P.h_elems + R.h_off + (int64_t)s * D);
#pragma unroll
        for (int c = 0; c < D / 2; ++c) {
            const float4 v = hrow[c];
            ar[2 * c] = v.x; ai[2 * c] = v.y; ar[2 * c + 1] = v.z; ai[2 * c + 1] = v.w;
        }
    } else {
#pragma unroll
        for (int c = 0; c < D; ++c) { ar[c] = 0.f; ai[c] = 0.f; }
    }
    const int64_t mbase = (int64_t)inst * P.msg_elems;
    const int64_t rbase = (int64_t)inst * P.rho_elems;
    for (int q = R.child_begin; q < R.child_end; ++q) {
        const PairInfo pi = P.child_info[q];
        const int M = pi.mask;
        const int Df = 1 << pi.kf;
        const int a = pext_bits(s, M);
        const int rest = s & ~M;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            if ((c & ~M) == rest) {
                const int x = a * Df + pext_bits(c, M);
                const float2 m = pass_entry(io, T, mbase + pi.off + x, rbase + pi.child_rho + x, false);
                ar[c] -= m.x;
                ai[c] -= m.y;
            }
        }
    }
    for (int q = R.parent_begin; q < R.parent_end; ++q) {
        const PairInfo pi = P.parent_info[q];
        if constexpr (D <= 8) {   // float4 gathers; at larger D the unrolled loads would crowd the registers
#pragma unroll
            for (int c = 0; c < D; c += 2) {
                const int64_t x = (int64_t)s * D + c;
                const float4 m = pass_entry2(io, T, mbase + pi.off + x, rbase + R.rho_off + x, true);
                ar[c] += m.x;
                ai[c] += m.y;
                ar[c + 1] += m.z;
                ai[c + 1] += m.w;
            }
        } else {
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const int64_t x = (int64_t)s * D + c;
                const float2 m = pass_entry(io, T, mbase + pi.off + x, rbase + R.rho_off + x, true);
                ar[c] += m.x;
                ai[c] += m.y;
            }
        }
    }
}

}  // namespace dev
}  // namespace lrh
