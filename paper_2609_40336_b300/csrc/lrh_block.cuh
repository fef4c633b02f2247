// Region pass for regions of 3 and 4 sites (D = 8, 16) in the Hermitian 2x2-block layout, sm_103a:
// device code shared by the per-class kernel (lrh_block.cu) and the one-launch / persistent
// drivers (lrh_kernels.cu).
//
// A group of D lanes owns one region (32 / D regions per warp).  theta lives in shared memory as
// the upper triangle of its D/2 x D/2 grid of 2x2 blocks (block (k, l), k <= l, holds rows 2k, 2k+1
// and columns 2l, 2l+1), so every Hermitian pair of entries is stored and rotated once.  A sweep
// of the cyclic two-sided Jacobi method runs D-1 rounds of the round-robin tournament with the
// pairs always in slots (2k, 2k+1); the tournament's slot permutation is applied by writing every
// rotated entry (i, j) to its next position (dst(i), dst(j)) (conjugated when that falls below the
// diagonal) in a second buffer.  The permutation is the same in every round, so each lane computes
// its source blocks and destination positions once.  Every round:
//   1. lanes k < D/2 take the diagonal block (k, k): the rotation (c, w) that zeroes its
//      off-diagonal entry and the two new diagonal entries (exact: the block becomes diagonal);
//   2. lanes update the D(D-2)/8 off-diagonal blocks, B' = J_k^H B J_l (two-sided, one pass);
//   3. lane s applies the column rotation and the tournament permutation to row s of V
//      (registers, compile-time indices, two register arrays used in turn), one round late, so
//      that step 1's dependent chain (computed by every lane, stored by lanes k < D/2) overlaps
//      V's independent FMAs in one basic block.
// The rotation parameters use the fast reciprocal / reciprocal square root (rot_fast).
// Arithmetic per round: 12 FMA-type instructions per stored entry of theta and 6 per entry of V,
// against 18 per row entry (both triangles of theta, plus V) in the lane-row layout.
// After the sweeps, the Gibbs state / ground projector, the partial traces and the values are
// formed as in the lane-row pass (same conventions, same outputs).
#pragma once
#include "lrh_device.cuh"
#include "lrh_internal.cuh"

#include <cstdint>

namespace lrh {
namespace blk {

using namespace dev;

// Placement of the 16 x 16 layout in shared memory.  A buffer holds 72 units of 16 bytes (unit
// u < 36: entries (0, 1) of block u; unit 36 + u: entries (2, 3)), spread over 144 unit slots
// (the buffers share their space with the W / rho staging, which needs twice as much), and the
// 28 off-diagonal blocks are dealt to the 32 (lane, j) positions of a region.  Both were chosen
// by a search (paper_2609_40336_b300/blk16_layout.py) that minimises the shared-memory
// wavefronts of a round: 64-bit stores are served per 16 lanes and 128-bit loads per 8, and two
// lanes hitting the same bank at different addresses cost one more wavefront; the search cut the
// modelled wavefronts of a round's block loads and stores from 43 to 31.
static __constant__ unsigned char kPhys16[72] = {30, 39, 76, 102, 131, 141, 42, 7, 95, 80, 33, 132, 49, 29, 26, 108, 90, 109, 59, 93, 47, 9, 113, 97, 46, 107, 64, 110, 32, 15, 35, 0, 22, 122, 140, 37, 78, 127, 56, 135, 14, 98, 61, 50, 23, 1, 2, 100, 48, 53, 69, 18, 123, 3, 124, 74, 115, 8, 72, 4, 126, 118, 27, 63, 101, 103, 133, 62, 57, 17, 129, 12};
// off-diagonal block (in (k, l) row order) of position j * 16 + lane; -1: repeats block 27
static __constant__ signed char kAssign16[32] = {18, -1, 22, 23, 14, 21, 6, 27, 4, 5, 10, 17, 9, 3, 7, 2, 8, 26, 15, 0, 25, 1, 11, 13, -1, 16, 24, 12, -1, -1, 19, 20};

template <int D>
struct Blk {
    static constexpr int n = D / 2;                  // pairs per round
    static constexpr int NB = n * (n + 1) / 2;       // stored blocks (k <= l)
    static constexpr int NOFF = n * (n - 1) / 2;     // off-diagonal blocks
    static constexpr int PER = (NOFF + D - 1) / D;   // off-diagonal blocks per lane
    static constexpr int LD = D + 2;                 // padded row stride of the W / rho staging
    static constexpr int SLOTS = D == 16 ? 144 : 2 * NB;   // 16-byte unit slots per buffer
    // one buffer: unit u < NB = entries (0, 1) of block u, unit NB + u = entries (2, 3), placed
    // at slot phys_unit<D>(u)
    static constexpr size_t buf_bytes = (size_t)SLOTS * 16;
    static constexpr size_t stage_bytes = (size_t)2 * D * LD * sizeof(float2);
    static constexpr size_t union_bytes = 2 * buf_bytes > stage_bytes ? 2 * buf_bytes : stage_bytes;
    static constexpr size_t per_group = union_bytes + 2 * n * sizeof(RotC<float>) + D * sizeof(float);
};

template <int D, int BLOCK>
struct BlkSmem {
    static constexpr size_t bytes = (BLOCK / D) * Blk<D>::per_group + 16;
};

// next slot of the entries in slot o (inverse of the tournament's rr_src)
__host__ __device__ constexpr int rr_dst(int o, int D) {
    return o == 0 ? 0 : (o == 1 ? 2 : ((o & 1) ? o - 2 : (o == D - 2 ? D - 1 : o + 2)));
}

template <int D>
__device__ __forceinline__ int bidx(int k, int l) { return k * (D / 2) - ((k * (k - 1)) >> 1) + (l - k); }

// slot of unit u
template <int D>
__device__ __forceinline__ int phys_unit(int u) {
    if constexpr (D == 16) return kPhys16[u];
    else return u;
}

// float2 index (within one buffer) of entry (i, j), i <= j
template <int D>
__device__ __forceinline__ int eidx(int i, int j) {
    const int e = ((i & 1) << 1) | (j & 1);
    return phys_unit<D>((e >> 1) * Blk<D>::NB + bidx<D>(i >> 1, j >> 1)) * 2 + (e & 1);
}

// off-diagonal block of position (j, lane) (in (k, l) row order) and whether the position owns it
// (positions without a block of their own repeat one: the same values to the same places)
template <int D>
__device__ __forceinline__ int assigned_block(int j, int lane, bool& own) {
    constexpr int NOFF = Blk<D>::NOFF;
    if constexpr (D == 16) {
        const int m = kAssign16[j * 16 + lane];
        own = m >= 0;
        return m >= 0 ? m : NOFF - 1;
    } else {
        const int m = lane + D * j;
        own = m < NOFF;
        return own ? m : NOFF - 1;
    }
}

// destination of entry (i, j), i <= j, after a round: its float2 index, negative (~index) when the
// entry lands below the diagonal and is stored conjugated
template <int D>
__device__ __forceinline__ int dest(int i, int j) {
    const int I = rr_dst(i, D), J = rr_dst(j, D);
    return I <= J ? eidx<D>(I, J) : ~eidx<D>(J, I);
}

// Rotation of pair (p, q) from a_pp, a_qq, a_pq (the same rotation as rot_params_d) and the two
// diagonal entries after it.  With h = a_qq - a_pp, den = |h| + sqrt(h^2 + 4 |a_pq|^2) and
// q = 2 / den: t = -sgn(h) q |a_pq|, c = 1 / sqrt(1 + t^2) = rsqrt(1 + q^2 |a_pq|^2),
// sigma = -sgn(h) q c, and t |a_pq| = -sgn(h) q |a_pq|^2, so |a_pq| itself is never needed:
// one square root, one reciprocal and one reciprocal square root.  The rotation is unitary when
// c^2 (1 + q^2 |a_pq|^2) = 1, whatever q is, so c gets one Newton step after the fast reciprocal
// square root (about 1 ulp, like the IEEE forms); the fast square root and reciprocal only
// perturb the angle, i.e. the pair's off-diagonal entry left before it is set to zero, an error
// of the order of the rounding of the entries themselves.
__device__ __forceinline__ void rot_fast(float app, float aqq, float br, float bi, RotC<float>& R, float2& dnew) {
    const float h = aqq - app;
    const float b2 = fmaf(br, br, bi * bi);
    const float r2 = fmaf(h, h, 4.f * b2);
    const float r = r2 > 0.f ? r2 * rsqrtf(r2) : 0.f;
    const float den = fabsf(h) + r;
    // den >= 2 |a_pq|; below 1e-18 the pair is diagonal at that absolute scale and is left as it
    // is (identity rotation); above it q^2 <= 4e36 cannot overflow and q^2 |a_pq|^2 <= 1
    const float q = den > 1e-18f ? __fdividef(2.f, den) : 0.f;
    const float sg = h >= 0.f ? 1.f : -1.f;
    const float x = fmaf(q * q, b2, 1.f);
    float c = rsqrtf(x);
    c = c * fmaf(-0.5f * x, c * c, 1.5f);   // Newton step: c^2 x = 1 to about one ulp
    const float sig = -sg * q * c;
    R.c = c;
    R.wr = sig * br;
    R.wi = sig * bi;
    R.pad = 0.f;
    const float tb = sg * q * b2;
    dnew.x = app - tb;
    dnew.y = aqq + tb;
}

// Row s of theta_e = h_e - sum_children 1 (x) m + sum_parents m, with the message entries of
// pass_entry (the same subtractions and additions in the same order as assemble_row_io, so the
// same values).  A child f of k_f sites touches D_f of the row's D entries: its message row
// a = pext(s, M_f) is gathered once (D_f entries, float4 loads) and subtracted at the columns
// rest | (the b-th submask of M_f) through the lane's row of `rowbuf` in shared memory, instead of
// an unrolled loop over all D columns that issues its loads for every column.
template <int D, int LD>
__device__ __forceinline__ void assemble_row_blk(const DevProblem& P, const RegionInfo& R, int inst, int s,
                                                 const PassIO& io, const Thetas& T, float2* rowbuf,
                                                 float (&ar)[D], float (&ai)[D]) {
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
    if (R.child_end > R.child_begin) {
        float4* row4 = reinterpret_cast<float4*>(rowbuf + s * LD);
        float2* row = rowbuf + s * LD;
#pragma unroll
        for (int c = 0; c < D / 2; ++c) row4[c] = make_float4(ar[2 * c], ai[2 * c], ar[2 * c + 1], ai[2 * c + 1]);
        for (int q = R.child_begin; q < R.child_end; ++q) {
            const PairInfo pi = P.child_info[q];
            const int M = pi.mask;
            const int Df = 1 << pi.kf;
            const int rest = s & ~M;
            const int64_t x0 = (int64_t)pext_bits(s, M) * Df;
            int sub = 0;   // submasks of M in increasing order: column rest | sub holds entry b
            for (int b = 0; b < Df; b += 2) {
                const float4 m = pass_entry2(io, T, mbase + pi.off + x0 + b, rbase + pi.child_rho + x0 + b, false);
                const int c0 = rest | sub;
                sub = ((sub | ~M) + 1) & M;
                const int c1 = rest | sub;
                sub = ((sub | ~M) + 1) & M;
                float2 v0 = row[c0], v1 = row[c1];
                v0.x -= m.x; v0.y -= m.y;
                v1.x -= m.z; v1.y -= m.w;
                row[c0] = v0;
                row[c1] = v1;
            }
        }
#pragma unroll
        for (int c = 0; c < D / 2; ++c) {
            const float4 v = row4[c];
            ar[2 * c] = v.x; ai[2 * c] = v.y; ar[2 * c + 1] = v.z; ai[2 * c + 1] = v.w;
        }
    }
    for (int q = R.parent_begin; q < R.parent_end; ++q) {
        const PairInfo pi = P.parent_info[q];
        if constexpr (D <= 8) {   // float4 gathers; at D = 16 the unrolled loads would crowd the registers
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

// Warm start of a region's eigensolve from a stored basis V (row s of V in (vr, vi), every lane
// of the group; the stored V is the previous pass's eigenvectors, unitary to FP32 rounding).
// One Newton-Schulz step restores unitarity to rounding, V <- V (3 I - V^H V) / 2, so that the
// defect does not build up over the passes; then theta <- V^H theta V, which has theta's
// eigenvalues and is nearly diagonal when theta moved little since V was formed.  Row s of theta
// comes in (ar, ai) and leaves as row s of V^H theta V; (vr, vi) leave as row s of the corrected
// V.  Staging: Va and Ga, two D x LD complex arrays of the group (the W / rho staging area).
// Every lane of the warp calls it (warp barriers inside).
template <int D, int LD>
__device__ __forceinline__ void warm_basis(float2* Va, float2* Ga, const int s, float (&ar)[D], float (&ai)[D],
                                           float (&vr)[D], float (&vi)[D]) {
    float xr[D], xi[D];
    auto put_row = [&](float2* A, const float (&yr)[D], const float (&yi)[D]) {
        float4* row = reinterpret_cast<float4*>(A + s * LD);
#pragma unroll
        for (int c = 0; c < D / 2; ++c) row[c] = make_float4(yr[2 * c], yi[2 * c], yr[2 * c + 1], yi[2 * c + 1]);
    };
    // x += (a_r + i a_i) * row c of A
    auto axpy_row = [&](const float2* A, const int c, const float a_r, const float a_i) {
        const float4* row = reinterpret_cast<const float4*>(A + c * LD);
#pragma unroll
        for (int t = 0; t < D / 2; ++t) {
            const float4 y = row[t];
            xr[2 * t] = fmaf(a_r, y.x, fmaf(-a_i, y.y, xr[2 * t]));
            xi[2 * t] = fmaf(a_r, y.y, fmaf(a_i, y.x, xi[2 * t]));
            xr[2 * t + 1] = fmaf(a_r, y.z, fmaf(-a_i, y.w, xr[2 * t + 1]));
            xi[2 * t + 1] = fmaf(a_r, y.w, fmaf(a_i, y.z, xi[2 * t + 1]));
        }
    };
    auto zero_x = [&]() {
#pragma unroll
        for (int t = 0; t < D; ++t) { xr[t] = 0.f; xi[t] = 0.f; }
    };
    // G = V^H V, row s: sum_c conj(V[c][s]) V[c][:]
    put_row(Va, vr, vi);
    __syncwarp();
    zero_x();
#pragma unroll 2
    for (int c = 0; c < D; ++c) {
        const float2 a = Va[c * LD + s];
        axpy_row(Va, c, a.x, -a.y);
    }
    put_row(Ga, xr, xi);
    __syncwarp();
    // V <- (3 V - V G) / 2, row s: 1.5 V[s][:] - 0.5 sum_c V[s][c] G[c][:]
    zero_x();
#pragma unroll 2
    for (int c = 0; c < D; ++c) {
        const float2 a = Va[s * LD + c];
        axpy_row(Ga, c, a.x, a.y);
    }
    {
        const float4* row = reinterpret_cast<const float4*>(Va + s * LD);
#pragma unroll
        for (int t = 0; t < D / 2; ++t) {
            const float4 y = row[t];
            xr[2 * t] = fmaf(1.5f, y.x, -0.5f * xr[2 * t]);
            xi[2 * t] = fmaf(1.5f, y.y, -0.5f * xi[2 * t]);
            xr[2 * t + 1] = fmaf(1.5f, y.z, -0.5f * xr[2 * t + 1]);
            xi[2 * t + 1] = fmaf(1.5f, y.w, -0.5f * xi[2 * t + 1]);
        }
    }
    __syncwarp();   // every lane has read Va (G, V G) and Ga (V G)
    put_row(Va, xr, xi);
    __syncwarp();
    // T = theta V, row s: sum_c theta[s][c] V[c][:] (theta's row in registers: unrolled)
    zero_x();
#pragma unroll
    for (int c = 0; c < D; ++c) axpy_row(Va, c, ar[c], ai[c]);
    put_row(Ga, xr, xi);
    __syncwarp();
    // V^H T, row s: sum_c conj(V[c][s]) T[c][:]
    zero_x();
#pragma unroll 2
    for (int c = 0; c < D; ++c) {
        const float2 a = Va[c * LD + s];
        axpy_row(Ga, c, a.x, -a.y);
    }
#pragma unroll
    for (int t = 0; t < D; ++t) { ar[t] = xr[t]; ai[t] = xi[t]; }
    {
        const float4* row = reinterpret_cast<const float4*>(Va + s * LD);
#pragma unroll
        for (int t = 0; t < D / 2; ++t) {
            const float4 y = row[t];
            vr[2 * t] = y.x; vi[2 * t] = y.y; vr[2 * t + 1] = y.z; vi[2 * t + 1] = y.w;
        }
    }
    __syncwarp();   // the staging is free again
}

template <int D, int BLOCK>
__device__ __forceinline__ void region_pass_blk_impl(const DevProblem& P, const PassIO& io,
                                                     const int32_t* __restrict__ cls, const int32_t count, const int k,
                                                     const int64_t tile) {
    using B = Blk<D>;
    constexpr int n = B::n, NB = B::NB, PER = B::PER, LD = B::LD;
    constexpr int G = BLOCK / D;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int g = threadIdx.x / D;
    const int s = threadIdx.x % D;
    unsigned char* base = smem_raw + g * B::per_group;
    float2* bufA = reinterpret_cast<float2*>(base);
    float2* bufB = bufA + 2 * B::SLOTS;
    RotC<float>* prm2 = reinterpret_cast<RotC<float>*>(base + B::union_bytes);   // [2][n] by round parity
    float* pw = reinterpret_cast<float*>(prm2 + 2 * n);
    __shared__ unsigned long long blk_sweeps, blk_capped;
    if (threadIdx.x == 0) { blk_sweeps = 0ull; blk_capped = 0ull; }

    const int64_t unit = tile * G + g;
    const bool valid = unit < (int64_t)P.n_inst * count;
    const int inst = valid ? (int)(unit / count) : 0;
    const int r = valid ? cls[unit % count] : 0;
    const bool nest = P.st->variant == 1;
    const int max_sweeps = P.st->max_sweeps;
    const Thetas T = pass_thetas(P, io);

    // ---- assemble row s (with a stored basis: of V^H theta V) and store its upper part (the
    //      matrix is exactly Hermitian)
    RegionInfo R;
    float vr[D], vi[D];   // row s of the starting basis (the identity, or the stored V)
    const bool warm = P.warm != nullptr && P.warm_off[k] >= 0 && !P.st->cold;   // uniform over the launch
    float4* wrow = (warm && valid)
        ? reinterpret_cast<float4*>(P.warm + P.warm_off[k] + unit * (int64_t)(D * D) + (int64_t)s * D)
        : nullptr;
    {
        float ar[D], ai[D];
        if (valid) {
            R = P.reg[r];
            assemble_row_blk<D, LD>(P, R, inst, s, io, T, reinterpret_cast<float2*>(base), ar, ai);
        } else {
            R = RegionInfo{-1, -1, 0, 0, 0, 0, 0};
#pragma unroll
            for (int c = 0; c < D; ++c) { ar[c] = 0.f; ai[c] = 0.f; }
        }
        __syncwarp();   // every lane is done with its staging row before the buffers are written
        if (wrow) {
#pragma unroll
            for (int c = 0; c < D / 2; ++c) {
                const float4 v = wrow[c];
                vr[2 * c] = v.x; vi[2 * c] = v.y; vr[2 * c + 1] = v.z; vi[2 * c + 1] = v.w;
            }
        } else {
#pragma unroll
            for (int c = 0; c < D; ++c) { vr[c] = c == s ? 1.f : 0.f; vi[c] = 0.f; }
        }
        if (warm) {
            float2* Va = reinterpret_cast<float2*>(base);
            warm_basis<D, LD>(Va, Va + D * LD, s, ar, ai, vr, vi);
        }
#pragma unroll
        for (int c = 0; c < D; ++c)
            if (c >= s) bufA[eidx<D>(s, c)] = make_float2(ar[c], c == s ? 0.f : ai[c]);
    }

    // ---- blocks and destinations of every lane position (the same in every round and for every
    //      region of the CTA): for position (j, lane), byte offsets of its block's two halves and
    //      of the rotations of the block's row and column pairs, the float2 indices of its four
    //      entries' next positions, +-1 for the entries stored conjugated, and whether the
    //      position owns the block
    __shared__ int4 tab_off[PER * D];
    __shared__ int4 tab_dst[PER * D];
    __shared__ float4 tab_sgn[PER * D];
    __shared__ int tab_own[PER * D];
    if (threadIdx.x < PER * D) {
        const int j = threadIdx.x / D, ls = threadIdx.x % D;
        bool own;
        int m = assigned_block<D>(j, ls, own), kq = 0;
        while (m >= n - 1 - kq) { m -= n - 1 - kq; ++kq; }
        const int lq = kq + 1 + m;
        const int bb = bidx<D>(kq, lq);
        tab_off[threadIdx.x] = make_int4(16 * phys_unit<D>(bb), 16 * phys_unit<D>(NB + bb), 16 * kq, 16 * lq);
        tab_own[threadIdx.x] = own ? 1 : 0;
        int d[4];
        float sg[4];
        for (int e = 0; e < 4; ++e) {
            const int x = dest<D>(2 * kq + (e >> 1), 2 * lq + (e & 1));
            d[e] = x < 0 ? ~x : x;
            sg[e] = x < 0 ? -1.f : 1.f;
        }
        tab_dst[threadIdx.x] = make_int4(d[0], d[1], d[2], d[3]);
        tab_sgn[threadIdx.x] = make_float4(sg[0], sg[1], sg[2], sg[3]);
    }
    __syncthreads();
    // the same table in registers, packed (a round reads it without shared-memory traffic):
    // pk0 = unit slots of the block's two halves (bits 0-7, 8-15) and the byte offsets of its
    // row and column rotations (16-23, 24-31); pk1 / pk2 = float2 indices of the next positions
    // of entries 0, 1 / 2, 3 (bits 0-14, 16-30), bits 15 / 31 set when the entry is stored
    // conjugated
    uint32_t pk1[PER], pk2[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int4 dd = tab_dst[j * D + s];
        const float4 sg = tab_sgn[j * D + s];
        pk1[j] = (uint32_t)dd.x | (sg.x < 0.f ? 0x8000u : 0u) | ((uint32_t)dd.y << 16) | (sg.y < 0.f ? 0x80000000u : 0u);
        pk2[j] = (uint32_t)dd.z | (sg.z < 0.f ? 0x8000u : 0u) | ((uint32_t)dd.w << 16) | (sg.w < 0.f ? 0x80000000u : 0u);
    }
    // this lane's diagonal block: pair s mod (D/2) (lanes s >= D/2 compute a copy and store
    // nothing), and the next positions of its entries (never conjugated: 0 and 3 stay on the
    // diagonal, and entry 1 is written as zero)
    const int pp = s & (n - 1);
    const int sd0 = phys_unit<D>(bidx<D>(pp, pp)), sd1 = phys_unit<D>(NB + bidx<D>(pp, pp));
    const int d0 = dest<D>(2 * pp, 2 * pp), d3 = dest<D>(2 * pp + 1, 2 * pp + 1);
    const int d1x = dest<D>(2 * pp, 2 * pp + 1), d1 = d1x < 0 ? ~d1x : d1x;
    const float sg1 = d1x < 0 ? -1.f : 1.f;
    // Each region stops at its own test; while other regions of the warp still sweep, a stopped
    // region runs identity rotations (every value kept exactly, only the tournament permutation
    // applied, which whole sweeps undo), so its result does not depend on its warp neighbours.
    bool active = true;

    // V takes each round's rotations one round late (so that their dependent chain overlaps V's
    // independent FMAs); it starts as the starting basis with its columns in inverse tournament
    // order, so that the first, rotation-free step (y[c] = x[rr_src(c)]) restores it
    {
        float tr_[D], ti_[D];
#pragma unroll
        for (int c = 0; c < D; ++c) { tr_[c] = vr[c]; ti_[c] = vi[c]; }
#pragma unroll
        for (int c = 0; c < D; ++c) { vr[rr_src(c, D)] = tr_[c]; vi[rr_src(c, D)] = ti_[c]; }
    }
    if (s < 2 * n) prm2[s] = RotC<float>{1.f, 0.f, 0.f, 0.f};
    __syncwarp();

    // squared Frobenius norms: off-diagonal part (both triangles) and whole matrix
    auto sums = [&](const float2* cur, float& off, float& all) {
        const float4* c4 = reinterpret_cast<const float4*>(cur);
        float o = 0.f, dg = 0.f;
#pragma unroll 1
        for (int j = 0; j < PER; ++j)
            if (tab_own[j * D + s]) {
                const int4 of = tab_off[j * D + s];
                const float4 h0 = c4[of.x >> 4], h1 = c4[of.y >> 4];
                o += h0.x * h0.x + h0.y * h0.y + h0.z * h0.z + h0.w * h0.w + h1.x * h1.x + h1.y * h1.y + h1.z * h1.z + h1.w * h1.w;
            }
        if (s < n) {
            const float4 h0 = c4[sd0], h1 = c4[sd1];
            o += h0.z * h0.z + h0.w * h0.w;
            dg = h0.x * h0.x + h1.z * h1.z;
        }
        off = 2.f * group_sum<D>(o);
        all = off + group_sum<D>(dg);
    };

    // V step: the rotations `pr` on row s of V (x), then the tournament permutation into y
    auto vstep = [&](const RotC<float>* pr, float (&xr)[D], float (&xi)[D], float (&yr)[D], float (&yi)[D]) {
#pragma unroll
        for (int q = 0; q < n; ++q) {
            const RotC<float> Q = pr[q];
            mix_cols(xr[2 * q], xi[2 * q], xr[2 * q + 1], xi[2 * q + 1], Q.c, Q.wr, Q.wi);
        }
#pragma unroll
        for (int c = 0; c < D; ++c) { yr[c] = xr[rr_src(c, D)]; yi[c] = xi[rr_src(c, D)]; }
    };

    // one round with parity par: rotations from the diagonal blocks of `cur` into prm2[par], the
    // delayed V step with prm2[par ^ 1] (x into y), then every off-diagonal block into `nxt` at
    // its next position
    auto round = [&](const float2* cur, float2* nxt, int par, float (&xr)[D], float (&xi)[D], float (&yr)[D],
                     float (&yi)[D]) {
        const float4* c4 = reinterpret_cast<const float4*>(cur);
        const unsigned char* cb = reinterpret_cast<const unsigned char*>(cur);
        RotC<float>* pc = prm2 + n * par;
        const unsigned char* pb = reinterpret_cast<const unsigned char*>(pc);
        {
            const float4 h0 = c4[sd0], h1 = c4[sd1];
            RotC<float> Rk;
            float2 dn;
            rot_fast(h0.x, h1.z, h0.z, h0.w, Rk, dn);
            float2 b1 = make_float2(0.f, 0.f);
            if (!active) {
                Rk = RotC<float>{1.f, 0.f, 0.f, 0.f};
                dn = make_float2(h0.x, h1.z);
                b1 = make_float2(h0.z, sg1 * h0.w);
            }
            if (s < n) {
                pc[s] = Rk;
                nxt[d0] = make_float2(dn.x, 0.f);
                nxt[d3] = make_float2(dn.y, 0.f);
                nxt[d1] = b1;
            }
        }
        vstep(prm2 + n * (par ^ 1), xr, xi, yr, yi);
        __syncwarp();
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            {   // a lane without a j-th block repeats a valid block: the same values to the same
                // places, and the round stays one basic block (loads of both blocks in flight)
                const uint32_t w1 = pk1[j], w2 = pk2[j];
                const int4 of = tab_off[j * D + s];
                const float4 h0 = *reinterpret_cast<const float4*>(cb + of.x);
                const float4 h1 = *reinterpret_cast<const float4*>(cb + of.y);
                float2 b00 = make_float2(h0.x, h0.y), b01 = make_float2(h0.z, h0.w);
                float2 b10 = make_float2(h1.x, h1.y), b11 = make_float2(h1.z, h1.w);
                const RotC<float> K = *reinterpret_cast<const RotC<float>*>(pb + of.z);
                const RotC<float> Lr = *reinterpret_cast<const RotC<float>*>(pb + of.w);
                two_sided<float>(b00, b01, b10, b11, K, Lr);
                // conjugation: flip the sign bit of the imaginary part
                auto cj = [](float y, uint32_t bit31) { return __int_as_float(__float_as_int(y) ^ (int)(bit31 & 0x80000000u)); };
                nxt[w1 & 0x7fffu] = make_float2(b00.x, cj(b00.y, w1 << 16));
                nxt[(w1 >> 16) & 0x7fffu] = make_float2(b01.x, cj(b01.y, w1));
                nxt[w2 & 0x7fffu] = make_float2(b10.x, cj(b10.y, w2 << 16));
                nxt[(w2 >> 16) & 0x7fffu] = make_float2(b11.x, cj(b11.y, w2));
            }
        }
        __syncwarp();
    };

    float off2, norm2;
    float2* cur = bufA;
    float2* nxt = bufB;
    sums(cur, off2, norm2);
    const float thresh = 1e-12f * norm2;
    int sweeps = 0, par = 0;
    float ur[D], ui[D];
    for (bool first = true;; first = false) {
        if (!first) {
            float o2, a2;
            sums(cur, o2, a2);
            if (active) { off2 = o2; norm2 = a2; }
        }
        if (active) active = !((off2 <= thresh) || (sweeps >= max_sweeps));
        if (!__any_sync(kFull, active)) break;
        if (active) ++sweeps;
#pragma unroll 1
        for (int rd = 0; rd + 1 < D - 1; rd += 2) {
            round(cur, nxt, par, vr, vi, ur, ui);
            round(nxt, cur, par ^ 1, ur, ui, vr, vi);
        }
        round(cur, nxt, par, vr, vi, ur, ui);   // D - 1 rounds per sweep is odd
        { float2* t = cur; cur = nxt; nxt = t; }
        par ^= 1;
#pragma unroll
        for (int c = 0; c < D; ++c) { vr[c] = ur[c]; vi[c] = ui[c]; }
    }
    // the last round's rotations (or, with no sweep, the initial permutation) complete V
    vstep(prm2 + n * (par ^ 1), vr, vi, ur, ui);
#pragma unroll
    for (int c = 0; c < D; ++c) { vr[c] = ur[c]; vi[c] = ui[c]; }
    // the slots are back in natural order: lambda_s on the diagonal, row s of V in (vr, vi),
    // stored as the next pass's starting basis (the identity when the region's V is not finite,
    // so that a non-finite input does not outlive the pass that saw it)
    if (warm) {
        bool fin = true;
#pragma unroll
        for (int c = 0; c < D; ++c) fin = fin && isfinite(vr[c]) && isfinite(vi[c]);
        const bool bad = group_sum<D>(fin ? 0.f : 1.f) > 0.f;   // every lane of the warp
        if (wrow) {
#pragma unroll
            for (int c = 0; c < D / 2; ++c)
                wrow[c] = bad ? make_float4(2 * c == s ? 1.f : 0.f, 0.f, 2 * c + 1 == s ? 1.f : 0.f, 0.f)
                              : make_float4(vr[2 * c], vi[2 * c], vr[2 * c + 1], vi[2 * c + 1]);
        }
    }
    const float lam = cur[eidx<D>(s, s)].x;
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
    __syncwarp();   // every lane has read its diagonal before the staging reuses the buffers
    pw[s] = sqrtf(wgt);
    float2* Wb = reinterpret_cast<float2*>(base);
    float2* Rb = Wb + D * LD;
    __syncwarp();
    // W = V diag(sqrt(p)); rho = W W^dagger, row s per lane (ur, ui reused)
#pragma unroll
    for (int c = 0; c < D; ++c) { const float q = pw[c]; ur[c] = vr[c] * q; ui[c] = vi[c] * q; }
    {
        float4* wrow = reinterpret_cast<float4*>(Wb + s * LD);
#pragma unroll
        for (int c = 0; c < D / 2; ++c) wrow[c] = make_float4(ur[2 * c], ui[2 * c], ur[2 * c + 1], ui[2 * c + 1]);
    }
    __syncwarp();
    // entry (s, j) for j = s + d mod D, d = 0..D/2: every unordered pair once (d = D/2 from the
    // lower of its two rows), D/2 + 1 entries per lane instead of a triangle's D - s
    for (int d = 0; d <= D / 2; ++d) {
        if (d == D / 2 && s >= D / 2) break;
        const int j = (s + d) & (D - 1);
        const float4* wj = reinterpret_cast<const float4*>(Wb + j * LD);
        float accr = 0.f, acci = 0.f;
#pragma unroll
        for (int c = 0; c < D / 2; ++c) {
            const float4 x = wj[c];
            accr += ur[2 * c] * x.x + ui[2 * c] * x.y;
            acci += ui[2 * c] * x.x - ur[2 * c] * x.y;
            accr += ur[2 * c + 1] * x.z + ui[2 * c + 1] * x.w;
            acci += ui[2 * c + 1] * x.z - ur[2 * c + 1] * x.w;
        }
        Rb[s * LD + j] = make_float2(accr, d == 0 ? 0.f : acci);
        if (d > 0) Rb[j * LD + s] = make_float2(accr, -acci);   // exactly Hermitian
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
    __syncthreads();
    if (valid && s == 0) {
        atomicAdd(&blk_sweeps, (unsigned long long)sweeps);
        if (off2 > thresh) atomicAdd(&blk_capped, 1ull);
    }
    __syncthreads();
    if (threadIdx.x == 0 && blk_sweeps) atomicAdd(&P.sweeps[k], blk_sweeps);
    if (threadIdx.x == 0 && blk_capped) atomicAdd(&P.capped[k], blk_capped);
}


// ---------------------------------------------------------------------------------------------
// One warp per 16 x 16 region (launch shape LRH_SHAPE_WARP16): the same block layout, rotations
// and tournament as region_pass_blk_impl<16>, with the work spread over 32 lanes.
//   * lane j < 28 owns off-diagonal block j for the whole eigensolve, so its source offset,
//     destinations and signs stay in registers (lanes 28..31 repeat block 27: the same values
//     to the same places, no divergence);
//   * lane 2 r + h owns half h of row r of V (8 columns; the tournament moves one entry across
//     the half-row boundary per round: one shuffle pair);
//   * every lane computes the rotation of pair (lane mod 8) (lanes 0..7 store it), and V takes
//     each round's rotations one round late, so the rotation's dependent chain overlaps V's
//     independent FMAs in one basic block.  V starts as the identity with its columns in the
//     inverse tournament order, so that the first (delayed) step, which only permutes, yields
//     the identity; one more step after the last round applies the last rotations.
// Rotations, block updates and V updates are those of region_pass_blk_impl<16> in the same
// order; results agree with it to rounding (a few operations are ordered differently).
struct W16 {
    static constexpr int D = 16, n = 8, NB = 36, NOFF = 28, LD = D + 2;
    static constexpr size_t union_bytes = Blk<16>::union_bytes;
    static constexpr size_t per_group = union_bytes + 2 * n * sizeof(RotC<float>) + D * sizeof(float);
};

template <int BLOCK>
struct W16Smem {
    static constexpr size_t bytes = (BLOCK / 32) * W16::per_group + 16;
};

template <int BLOCK>
__device__ __forceinline__ void region_pass_w16_impl(const DevProblem& P, const PassIO& io,
                                                     const int32_t* __restrict__ cls, const int32_t count, const int k,
                                                     const int64_t tile) {
    constexpr int D = 16, n = 8, NB = 36, NOFF = 28, LD = W16::LD, H = D / 2;
    constexpr int G = BLOCK / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int g = threadIdx.x >> 5;
    const int L = threadIdx.x & 31;
    const int s = L & (D - 1);            // row of theta / rho for lanes 0..15
    unsigned char* base = smem_raw + g * W16::per_group;
    float2* bufA = reinterpret_cast<float2*>(base);
    float2* bufB = bufA + 2 * Blk<16>::SLOTS;
    RotC<float>* prm2 = reinterpret_cast<RotC<float>*>(base + W16::union_bytes);   // [2][n] by round parity
    float* pw = reinterpret_cast<float*>(prm2 + 2 * n);
    __shared__ unsigned long long blk_sweeps, blk_capped;
    if (threadIdx.x == 0) { blk_sweeps = 0ull; blk_capped = 0ull; }

    const int64_t unit = tile * G + g;
    const bool valid = unit < (int64_t)P.n_inst * count;
    const int inst = valid ? (int)(unit / count) : 0;
    const int r = valid ? cls[unit % count] : 0;
    const bool nest = P.st->variant == 1;
    const int max_sweeps = P.st->max_sweeps;
    const Thetas T = pass_thetas(P, io);

    // ---- assemble: lanes 0..15 build row s and store its upper part
    const RegionInfo R = valid ? P.reg[r] : RegionInfo{-1, -1, 0, 0, 0, 0, 0};
    if (L < D) {
        float ar[D], ai[D];
        if (valid) {
            assemble_row_io<D>(P, R, inst, s, io, T, ar, ai);
        } else {
#pragma unroll
            for (int c = 0; c < D; ++c) { ar[c] = 0.f; ai[c] = 0.f; }
        }
#pragma unroll
        for (int c = 0; c < D; ++c)
            if (c >= s) bufA[eidx<D>(s, c)] = make_float2(ar[c], c == s ? 0.f : ai[c]);
    }
    if (L < 2 * n) prm2[L] = RotC<float>{1.f, 0.f, 0.f, 0.f};   // the "previous" rotations of round 0

    // ---- this lane's off-diagonal block (the same in every round)
    int boff, boff1, koff, loff, dd[4];
    float sg[4];
    {
        int m = L < NOFF ? L : NOFF - 1, kq = 0;
        while (m >= n - 1 - kq) { m -= n - 1 - kq; ++kq; }
        const int lq = kq + 1 + m;
        boff = 16 * phys_unit<D>(bidx<D>(kq, lq));
        boff1 = 16 * phys_unit<D>(NB + bidx<D>(kq, lq));
        koff = 16 * kq;
        loff = 16 * lq;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int x = dest<D>(2 * kq + (e >> 1), 2 * lq + (e & 1));
            dd[e] = x < 0 ? ~x : x;
            sg[e] = x < 0 ? -1.f : 1.f;
        }
    }
    // this lane's diagonal block (pair L mod 8) and the next positions of its entries
    const int pp = L & (n - 1);
    const int sd0 = phys_unit<D>(bidx<D>(pp, pp)), sd1 = phys_unit<D>(NB + bidx<D>(pp, pp));
    const int d0 = dest<D>(2 * pp, 2 * pp), d3 = dest<D>(2 * pp + 1, 2 * pp + 1);
    const int d1x = dest<D>(2 * pp, 2 * pp + 1), d1 = d1x < 0 ? ~d1x : d1x;
    // V: lane L holds half hh of row vrow, columns 8 hh .. 8 hh + 7, starting as the identity with
    // its columns in inverse tournament order (the first V step, y[c] = x[rr_src(c)], restores it)
    const int vrow = L >> 1, hh = L & 1;
    float vr[H], vi[H], ur[H], ui[H];
#pragma unroll
    for (int c = 0; c < H; ++c) { vr[c] = (H * hh + c == rr_src(vrow, D)) ? 1.f : 0.f; vi[c] = 0.f; }
    __syncwarp();

    auto sums = [&](const float2* cur, float& off, float& all) {
        const unsigned char* cb = reinterpret_cast<const unsigned char*>(cur);
        const float4* c4 = reinterpret_cast<const float4*>(cur);
        float o = 0.f, dg = 0.f;
        if (L < NOFF) {
            const float4 h0 = *reinterpret_cast<const float4*>(cb + boff);
            const float4 h1 = *reinterpret_cast<const float4*>(cb + boff1);
            o = h0.x * h0.x + h0.y * h0.y + h0.z * h0.z + h0.w * h0.w + h1.x * h1.x + h1.y * h1.y + h1.z * h1.z + h1.w * h1.w;
        }
        if (L < n) {
            const float4 h0 = c4[sd0], h1 = c4[sd1];
            o += h0.z * h0.z + h0.w * h0.w;
            dg = h0.x * h0.x + h1.z * h1.z;
        }
        off = 2.f * group_sum<32>(o);
        all = off + group_sum<32>(dg);
    };

    // V step: the rotations `pr` on this lane's 4 column pairs, then the tournament permutation into
    // (yr, yi); one complex entry crosses between the two halves of a row (half 0 sends column 6,
    // half 1 sends column 9)
    auto vstep = [&](const RotC<float>* pr, float (&xr)[H], float (&xi)[H], float (&yr)[H], float (&yi)[H]) {
        const RotC<float>* ph = pr + 4 * hh;
#pragma unroll
        for (int q = 0; q < H / 2; ++q) {
            const RotC<float> Q = ph[q];
            mix_cols(xr[2 * q], xi[2 * q], xr[2 * q + 1], xi[2 * q + 1], Q.c, Q.wr, Q.wi);
        }
        const float sr = hh ? xr[1] : xr[6], si = hh ? xi[1] : xi[6];
        const float rr = __shfl_xor_sync(kFull, sr, 1), ri = __shfl_xor_sync(kFull, si, 1);
        // half 0: [x0, x3, x1, x5, x2, x7, x4, recv];  half 1: [recv, x3, x0, x5, x2, x7, x4, x6]
        yr[0] = hh ? rr : xr[0];  yi[0] = hh ? ri : xi[0];
        yr[1] = xr[3];            yi[1] = xi[3];
        yr[2] = hh ? xr[0] : xr[1]; yi[2] = hh ? xi[0] : xi[1];
        yr[3] = xr[5];            yi[3] = xi[5];
        yr[4] = xr[2];            yi[4] = xi[2];
        yr[5] = xr[7];            yi[5] = xi[7];
        yr[6] = xr[4];            yi[6] = xi[4];
        yr[7] = hh ? xr[6] : rr;  yi[7] = hh ? xi[6] : ri;
    };

    // one round with parity par: rotations from the diagonal blocks of `cur` into prm2[par], the
    // delayed V step with prm2[par ^ 1], then every off-diagonal block into `nxt`
    auto round = [&](const float2* cur, float2* nxt, int par, float (&xr)[H], float (&xi)[H], float (&yr)[H],
                     float (&yi)[H]) {
        const float4* c4 = reinterpret_cast<const float4*>(cur);
        const unsigned char* cb = reinterpret_cast<const unsigned char*>(cur);
        RotC<float>* pc = prm2 + n * par;
        {
            const float4 h0 = c4[sd0], h1 = c4[sd1];
            RotC<float> Rk;
            float2 dn;
            rot_fast(h0.x, h1.z, h0.z, h0.w, Rk, dn);
            if (L < n) {
                pc[L] = Rk;
                nxt[d0] = make_float2(dn.x, 0.f);
                nxt[d3] = make_float2(dn.y, 0.f);
                nxt[d1] = make_float2(0.f, 0.f);
            }
        }
        vstep(prm2 + n * (par ^ 1), xr, xi, yr, yi);
        __syncwarp();
        {
            const unsigned char* pb = reinterpret_cast<const unsigned char*>(pc);
            const float4 h0 = *reinterpret_cast<const float4*>(cb + boff);
            const float4 h1 = *reinterpret_cast<const float4*>(cb + boff1);
            float2 b00 = make_float2(h0.x, h0.y), b01 = make_float2(h0.z, h0.w);
            float2 b10 = make_float2(h1.x, h1.y), b11 = make_float2(h1.z, h1.w);
            const RotC<float> K = *reinterpret_cast<const RotC<float>*>(pb + koff);
            const RotC<float> Lr = *reinterpret_cast<const RotC<float>*>(pb + loff);
            two_sided<float>(b00, b01, b10, b11, K, Lr);
            nxt[dd[0]] = make_float2(b00.x, sg[0] * b00.y);
            nxt[dd[1]] = make_float2(b01.x, sg[1] * b01.y);
            nxt[dd[2]] = make_float2(b10.x, sg[2] * b10.y);
            nxt[dd[3]] = make_float2(b11.x, sg[3] * b11.y);
        }
        __syncwarp();
    };

    float off2, norm2;
    float2* cur = bufA;
    float2* nxt = bufB;
    sums(cur, off2, norm2);
    const float thresh = 1e-12f * norm2;
    int sweeps = 0, par = 0;
    for (;;) {
        if (sweeps > 0) sums(cur, off2, norm2);
        const bool done = (off2 <= thresh) || (sweeps >= max_sweeps);
        if (__all_sync(kFull, done)) break;
        ++sweeps;
#pragma unroll 1
        for (int rd = 0; rd + 1 < D - 1; rd += 2) {
            round(cur, nxt, par, vr, vi, ur, ui);
            round(nxt, cur, par ^ 1, ur, ui, vr, vi);
        }
        round(cur, nxt, par, vr, vi, ur, ui);   // D - 1 rounds per sweep is odd
        { float2* t = cur; cur = nxt; nxt = t; }
        par ^= 1;
#pragma unroll
        for (int c = 0; c < H; ++c) { vr[c] = ur[c]; vi[c] = ui[c]; }
    }
    // the last rounds' rotations (or, with no sweep, the initial permutation) complete V
    vstep(prm2 + n * (par ^ 1), vr, vi, ur, ui);
    // the slots are back in natural order: lambda_s on the diagonal, half hh of row vrow of V in (ur, ui)
    const float lam = cur[eidx<D>(s, s)].x;
    const float lmin = group_min<16>(lam);
    float wgt, F;
    if (nest) {
        const float beta = (float)P.st->beta;
        const float e = expf(-beta * (lam - lmin));
        const float Z = group_sum<16>(e);
        wgt = e / Z;
        F = lmin - logf(Z) / beta;
    } else {
        const float tau = (float)P.st->degen_tol * fmaxf(1.0f, sqrtf(norm2));
        const float in = (lam - lmin <= tau) ? 1.0f : 0.0f;
        const float m = group_sum<16>(in);
        wgt = in / m;
        F = lmin;
    }
    __syncwarp();   // every lane has read its diagonal before the staging reuses the buffers
    if (L < D) pw[s] = sqrtf(wgt);
    float2* Wb = reinterpret_cast<float2*>(base);
    float2* Rb = Wb + D * LD;
    __syncwarp();
    {   // W = V diag(sqrt(p)): this lane's half row
        float4* wrow = reinterpret_cast<float4*>(Wb + vrow * LD + H * hh);
#pragma unroll
        for (int c = 0; c < H / 2; ++c) {
            const float q0 = pw[H * hh + 2 * c], q1 = pw[H * hh + 2 * c + 1];
            wrow[c] = make_float4(ur[2 * c] * q0, ui[2 * c] * q0, ur[2 * c + 1] * q1, ui[2 * c + 1] * q1);
        }
    }
    __syncwarp();
    if (L < D) {   // rho = W W^dagger, upper triangle of row s (lanes 0..15)
        float wr_[D], wi_[D];
        {
            const float4* ws = reinterpret_cast<const float4*>(Wb + s * LD);
#pragma unroll
            for (int c = 0; c < D / 2; ++c) {
                const float4 x = ws[c];
                wr_[2 * c] = x.x; wi_[2 * c] = x.y; wr_[2 * c + 1] = x.z; wi_[2 * c + 1] = x.w;
            }
        }
        for (int j = s; j < D; ++j) {
            const float4* wj = reinterpret_cast<const float4*>(Wb + j * LD);
            float accr = 0.f, acci = 0.f;
#pragma unroll
            for (int c = 0; c < D / 2; ++c) {
                const float4 x = wj[c];
                accr += wr_[2 * c] * x.x + wi_[2 * c] * x.y;
                acci += wi_[2 * c] * x.x - wr_[2 * c] * x.y;
                accr += wr_[2 * c + 1] * x.z + wi_[2 * c + 1] * x.w;
                acci += wi_[2 * c + 1] * x.z - wr_[2 * c + 1] * x.w;
            }
            Rb[s * LD + j] = make_float2(accr, j == s ? 0.f : acci);
            if (j > s) Rb[j * LD + s] = make_float2(accr, -acci);   // exactly Hermitian
        }
    }
    __syncwarp();
    if (valid && L < D) {
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
    __syncthreads();
    if (valid && L == 0) {
        atomicAdd(&blk_sweeps, (unsigned long long)sweeps);
        if (off2 > thresh) atomicAdd(&blk_capped, 1ull);
    }
    __syncthreads();
    if (threadIdx.x == 0 && blk_sweeps) atomicAdd(&P.sweeps[k], blk_sweeps);
    if (threadIdx.x == 0 && blk_capped) atomicAdd(&P.capped[k], blk_capped);
}

}  // namespace blk
}  // namespace lrh
