// CTA-level region pass for D = 64 and D = 128 (regions of 6 and 7 sites), sm_103a.
//
// One CTA owns one region.  theta lives in shared memory: in the FP32 pass as the upper triangle
// of a row-padded D x (D+1) array with permuted indices, so that a warp's accesses fall on
// distinct banks (130 KB at D = 128), in the FP64 certification as a packed upper triangle
// (D(D+1)/2 complex entries: 132 KB at D = 128).  A sweep of the cyclic two-sided Jacobi
// method runs D-1 rounds of the round-robin tournament; instead of moving matrix entries, a
// slot -> index map (two small arrays in shared memory) is rotated each round.  Every round:
//   1. D/2 threads compute the rotation (c, w) of the pair in slots (2k, 2k+1);
//   2. the 2x2 blocks (k <= l) of the D/2 x D/2 block grid are updated in ONE pass,
//      B' = J_k^H B J_l: the blocks partition the unordered index pairs, so no two threads
//      touch the same entry and no second pass (row vs column) is needed;
//   3. V (in registers, 4 threads per row, columns in slot order) gets the column rotation
//      and then the tournament's column permutation, which moves one complex value across
//      each chunk boundary (two shuffles between the lanes holding neighbouring chunks).
// The Gibbs / ground state rho = W W^dagger, W = V diag(sqrt p), is formed either on the FP32
// cores from W^T staged in the same shared-memory buffer, with register tiles, or on the tensor
// cores (tcgen05, below); then made exactly Hermitian, traced onto the children and written out.  The FP64 certification kernel reuses the Jacobi part
// (no V) to return lambda_min.
#include "lrh_device.cuh"
#include "lrh_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdint>

namespace lrh {

namespace {

using dev::RotC;
using dev::rot_params_d;
using dev::two_sided;
using dev::kdd;
constexpr unsigned kFull = 0xffffffffu;

__host__ __device__ constexpr int rr_src_c(int s, int D) {
    return s == 0 ? 0 : (s == 2 ? 1 : ((s & 1) == 0 ? s - 2 : (s == D - 1 ? D - 2 : s + 2)));
}

__device__ __forceinline__ int pext8(int x, int m) {
    int r = 0, k = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b)
        if ((m >> b) & 1) { r |= ((x >> b) & 1) << k; ++k; }
    return r;
}

__device__ __forceinline__ int pdep8(int x, int m) {
    int r = 0, k = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b)
        if ((m >> b) & 1) { r |= ((x >> k) & 1) << b; ++k; }
    return r;
}

template <typename T> struct V2;
template <> struct V2<float> { using t = float2; };
template <> struct V2<double> { using t = double2; };



__device__ __forceinline__ int tri(int i, int j, int D) { return i * D - ((i * (i - 1)) >> 1) + (j - i); }

// Hermitian matrix in shared memory as a packed upper triangle (FP64 certification).
template <typename T>
struct Packed {
    using C2 = typename V2<T>::t;
    using Real = T;
    C2* a;
    int D;
    __device__ __forceinline__ int sig(int j) const { return j; }
    __device__ __forceinline__ C2 get(int i, int j) const {
        if (i <= j) return a[tri(i, j, D)];
        C2 v = a[tri(j, i, D)];
        v.y = -v.y;
        return v;
    }
    __device__ __forceinline__ void set(int i, int j, C2 v) const {
        if (i <= j) { a[tri(i, j, D)] = v; } else { v.y = -v.y; a[tri(j, i, D)] = v; }
    }
    __device__ __forceinline__ C2 dget(int i) const { return a[tri(i, i, D)]; }
    __device__ __forceinline__ void dset(int i, C2 v) const { a[tri(i, i, D)] = v; }
    // sums of |a_ij|^2 over the strict upper triangle and over the diagonal (summed separately:
    // the off-diagonal mass must not come out of a difference of two large sums)
    template <int NT>
    __device__ __forceinline__ void sums(T& offd, T& diag) const {
        offd = T(0); diag = T(0);
        for (int e = threadIdx.x; e < D * D; e += NT) {
            const int i = e / D, j = e - (e / D) * D;
            if (i < j) { const C2 v = a[tri(i, j, D)]; offd += v.x * v.x + v.y * v.y; }
        }
        for (int i = threadIdx.x; i < D; i += NT) { const C2 v = a[tri(i, i, D)]; diag += v.x * v.x + v.y * v.y; }
    }
};

// Hermitian matrix in shared memory for the FP32 pass: the upper triangle of a D x (D+1)
// row-padded array.  Logical index j is stored at position sig(j) = (j >> 1) + (j & 1) D/2 (rows
// and columns alike) and the Jacobi slot map holds positions; entry (i, j) of positions lives
// at (min, max), so its word address is congruent to 2 (i + j) modulo 32 banks whichever triangle
// it belongs to.  The tournament's slots hold positions that step by 1 from one slot pair to the
// next, so a warp's accesses fall on consecutive banks; no mirror writes are needed.
// get/set/dget/dset take positions.
template <typename T>
struct Full {
    using C2 = typename V2<T>::t;
    using Real = T;
    C2* a;
    int D;
    __device__ __forceinline__ int sig(int j) const { return (j >> 1) + (j & 1) * (D >> 1); }
    __device__ __forceinline__ C2 get(int i, int j) const {
        const bool up = i <= j;
        C2 v = a[up ? i * (D + 1) + j : j * (D + 1) + i];
        if (!up) v.y = -v.y;
        return v;
    }
    __device__ __forceinline__ void set(int i, int j, C2 v) const {
        const bool up = i <= j;
        if (!up) v.y = -v.y;
        a[up ? i * (D + 1) + j : j * (D + 1) + i] = v;
    }
    __device__ __forceinline__ C2 dget(int i) const { return a[i * (D + 2)]; }
    __device__ __forceinline__ void dset(int i, C2 v) const { a[i * (D + 2)] = v; }
    // sums of |a_ij|^2 over the strict upper triangle and over the diagonal (summed separately:
    // the off-diagonal mass must not come out of a difference of two large sums)
    template <int NT>
    __device__ __forceinline__ void sums(T& offd, T& diag) const {
        offd = T(0);
        diag = T(0);
        for (int e = threadIdx.x; e < D * D; e += NT) {
            const int i = e / D, j = e - (e / D) * D;
            if (i <= j) {
                const C2 v = a[i * (D + 1) + j];
                const T m = v.x * v.x + v.y * v.y;
                if (i == j) diag += m; else offd += m;
            }
        }
    }
};

// Hermitian matrix too large for shared memory (D = 256): a packed upper triangle whose first NS
// entries live in shared memory and the rest in a global-memory scratch slot of this CTA (held in
// L2 while the CTA runs).  Positions are the logical indices (sig = identity), as for Packed.
// Global entries are read and written with plain loads and stores; the CTA barriers between
// Jacobi phases make them visible to the other threads of the CTA.
template <typename T>
struct Split {
    using C2 = typename V2<T>::t;
    using Real = T;
    C2* s;     // entries [0, NS)
    C2* g;     // entries [NS, D (D + 1) / 2)
    int NS;
    int D;
    __device__ __forceinline__ int sig(int j) const { return j; }
    // separate shared and global accesses (a reference into either would force generic addressing)
    __device__ __forceinline__ C2 ld(int x) const {
        if (x < NS) return s[x];
        return g[x - NS];
    }
    __device__ __forceinline__ void st(int x, C2 v) const {
        if (x < NS) s[x] = v;
        else g[x - NS] = v;
    }
    __device__ __forceinline__ C2 get(int i, int j) const {
        if (i <= j) return ld(tri(i, j, D));
        C2 v = ld(tri(j, i, D));
        v.y = -v.y;
        return v;
    }
    __device__ __forceinline__ void set(int i, int j, C2 v) const {
        if (i <= j) { st(tri(i, j, D), v); } else { v.y = -v.y; st(tri(j, i, D), v); }
    }
    __device__ __forceinline__ C2 dget(int i) const { return ld(tri(i, i, D)); }
    __device__ __forceinline__ void dset(int i, C2 v) const { st(tri(i, i, D), v); }
    template <int NT>
    __device__ __forceinline__ void sums(T& offd, T& diag) const {
        offd = T(0); diag = T(0);
        for (int e = threadIdx.x; e < D * D; e += NT) {
            const int i = e / D, j = e - (e / D) * D;
            if (i < j) { const C2 v = ld(tri(i, j, D)); offd += v.x * v.x + v.y * v.y; }
        }
        for (int i = threadIdx.x; i < D; i += NT) { const C2 v = ld(tri(i, i, D)); diag += v.x * v.x + v.y * v.y; }
    }
};

// V rows in registers: a warp holds 8 rows x 4 column chunks, lane = 8 chunk + (row mod 8).
// The 8 lanes of a quarter-warp share one chunk, so the rotation parameters they read are one
// shared-memory address (a broadcast), and the neighbour chunk of the same row is 8 lanes away.
__device__ __forceinline__ int vrow_of(int t) { return (t >> 5) * 8 + (t & 7); }
__device__ __forceinline__ int vchunk_of(int t) { return (t >> 3) & 3; }

template <int NT, typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    T s = T(0);
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) s += red[i];
    return s;
}

// Rotation record of pair k: one pad record after every D/8 pairs (one V column chunk), so the
// four chunks' records that a warp reads in the same instruction fall on different banks.
template <int D>
__device__ __forceinline__ int prm_at(int k) { return k + k / (D / 8); }

template <int D> struct CtaCfg;
template <> struct CtaCfg<64> { static constexpr int NT = 256; static constexpr int TR = 4, TC = 4; };
template <> struct CtaCfg<128> { static constexpr int NT = 512; static constexpr int TR = 4, TC = 8; };
template <> struct CtaCfg<256> { static constexpr int NT = 1024; };

template <int D, typename T>
struct CtaSmem {
    static constexpr int n = D / 2;
    static constexpr int NB = n * (n + 1) / 2;
    static constexpr int NT = CtaCfg<D>::NT;
    static constexpr size_t tri_elems = (size_t)D * (D + 1) / 2;
    // FP32 kernel also stages W^T and rho (D x D) in the same buffer
    // FP32 pass: the Jacobi matrix (D x (D+1) complex), later the tensor-core operand chunks
    // (2 buffers x hi/lo x 2D rows x KC tf32) or the W^T / rho staging
    static constexpr size_t jac_bytes = sizeof(float2) * (size_t)D * (D + 1);
    static constexpr size_t tc_bytes = D == 128 ? (size_t)4 * (2 * D) * 32 * 4 : 0;   // 2 buffers x hi/lo
    static constexpr size_t buf_bytes_f = ((jac_bytes > tc_bytes ? jac_bytes : tc_bytes) + 127) / 128 * 128;
    static constexpr size_t buf_bytes_d = ((sizeof(double2) * tri_elems) + 15) / 16 * 16;
    static constexpr size_t buf_bytes = sizeof(T) == 4 ? buf_bytes_f : buf_bytes_d;
    static constexpr size_t off_prm = buf_bytes;
    static constexpr size_t off_idx = off_prm + sizeof(RotC<T>) * (n + 4);   // + one pad record per V chunk
    static constexpr size_t off_tab = off_idx + sizeof(int) * 2 * D;
    static constexpr size_t off_lam = off_tab + ((sizeof(unsigned short) * NB + 15) / 16 * 16);
    static constexpr size_t off_red = off_lam + sizeof(float) * 2 * D;
    static constexpr size_t off_mbar = (off_red + sizeof(double) * (NT / 32) + 15) / 16 * 16;   // 2 mbarriers + TMEM slot
    static constexpr size_t bytes = off_mbar + 32;
};

// Cyclic Jacobi on the Hermitian matrix behind accessor A; V (if WANT_V) holds row `row`,
// columns [chunk * W, chunk * W + W) in slot order.  Two barriers per round: after the rotation
// parameters, and after the block updates (the slot map is double-buffered and its next
// state written during the update phase).  Returns the sweeps run; `off_out` receives the
// squared Frobenius norm of the off-diagonal part left at exit.
// (Computing the next round's rotations inside the block updates, to save the first barrier,
// measured slower: the 64 parameter computations then fall on many warps, each of which runs
// the divisions and square roots for one lane, instead of two warps running them for all.)
template <int D, typename T, bool WANT_V, typename Acc>
__device__ int jacobi_cta(Acc A, RotC<T>* prm, int* idx0, int* idx1, const unsigned short* tab,
                          T* red, T (&vr)[D / 4], T (&vi)[D / 4], int max_sweeps, T tol2, T& norm2_out,
                          T& off_out) {
    using C2 = typename V2<T>::t;
    constexpr int NT = CtaCfg<D>::NT;
    constexpr int n = D / 2;
    // off-diagonal blocks (k < l) first, spread over all threads; the diagonal blocks (k = l,
    // about half the work each) go to the threads left idle by the last off-diagonal iteration
    constexpr int NOFF = n * (n - 1) / 2;
    constexpr int ITER = (NOFF + NT - 1) / NT;
    constexpr int IDLE = ITER * NT - NOFF;
    constexpr int DGT = IDLE > 0 ? IDLE : NT;         // threads that take diagonal blocks
    constexpr int DG0 = NT - DGT;                     // the first of them
    constexpr int JD0 = IDLE > 0 ? ITER - 1 : ITER;   // their first iteration without an off-diagonal block
    constexpr int NIT = JD0 + (n + DGT - 1) / DGT;
    constexpr int CH = 4;
    constexpr int W = D / CH;
    const int t = threadIdx.x;
    const int chunk = vchunk_of(t);
    T up, dg;
    A.template sums<NT>(up, dg);
    const T norm2 = T(2) * block_sum<NT>(up, red) + block_sum<NT>(dg, red);
    norm2_out = norm2;
    const T thresh = tol2 * norm2;
    int* ix = idx0;
    int* ixn = idx1;
    int sweeps = 0;
    for (;;) {
        A.template sums<NT>(up, dg);
        const T off = T(2) * block_sum<NT>(up, red);
        off_out = off;
        if (off <= thresh || sweeps >= max_sweeps) break;
        ++sweeps;
        for (int r = 0; r < D - 1; ++r) {
            if (t < n) {
                const int2 pq = reinterpret_cast<const int2*>(ix)[t];
                const auto b = A.get(pq.x, pq.y);
                C2 unused;
                rot_params_d<T>(A.dget(pq.x).x, A.dget(pq.y).x, b.x, b.y, prm[prm_at<D>(t)], unused);
            }
            __syncthreads();
            if (t < D) ixn[t] = ix[rr_src_c(t, D)];
            if (WANT_V) {
#pragma unroll
                for (int m = 0; m < W / 2; ++m) {
                    const RotC<T> Rk = prm[prm_at<D>((chunk * W) / 2 + m)];
                    T& pr = vr[2 * m]; T& pi = vi[2 * m]; T& qr = vr[2 * m + 1]; T& qi = vi[2 * m + 1];
                    const T npr = Rk.c * pr + (Rk.wr * qr + Rk.wi * qi);
                    const T npi = Rk.c * pi + (Rk.wr * qi - Rk.wi * qr);
                    const T nqr = Rk.c * qr - (Rk.wr * pr - Rk.wi * pi);
                    const T nqi = Rk.c * qi - (Rk.wr * pi + Rk.wi * pr);
                    pr = npr; pi = npi; qr = nqr; qi = nqi;
                }
            }
#pragma unroll 1
            for (int j = 0; j < NIT; ++j) {
                const int v = t + NT * j;
                if (v < NOFF) {
                    const int kl = tab[v];
                    const int kk = kl >> 8, ll = kl & 255;
                    const int2 pqk = reinterpret_cast<const int2*>(ix)[kk];
                    const int2 pql = reinterpret_cast<const int2*>(ix)[ll];
                    const int pk = pqk.x, qk = pqk.y, pl = pql.x, ql = pql.y;
                    auto b00 = A.get(pk, pl), b01 = A.get(pk, ql), b10 = A.get(qk, pl), b11 = A.get(qk, ql);
                    const RotC<T> K = prm[prm_at<D>(kk)];
                    const RotC<T> Lr = prm[prm_at<D>(ll)];
                    two_sided<T>(b00, b01, b10, b11, K, Lr);
                    A.set(pk, pl, b00); A.set(pk, ql, b01); A.set(qk, pl, b10); A.set(qk, ql, b11);
                } else {
                    const int kk = (t - DG0) + DGT * (j - JD0);
                    if (t >= DG0 && kk < n) {
                        const RotC<T> K = prm[prm_at<D>(kk)];
                        const int2 pq = reinterpret_cast<const int2*>(ix)[kk];
                        const int pk = pq.x, qk = pq.y;
                        auto b00 = A.dget(pk);
                        auto b11 = A.dget(qk);
                        auto b01 = A.get(pk, qk);
                        auto b10 = b01; b10.y = -b10.y;
                        b00.y = T(0); b11.y = T(0);
                        two_sided<T>(b00, b01, b10, b11, K, K);
                        b00.y = T(0); b11.y = T(0);
                        A.dset(pk, b00);
                        A.dset(qk, b11);
                        auto z = b01; z.x = T(0); z.y = T(0);
                        A.set(pk, qk, z);
                    }
                }
            }
            if (WANT_V) {
                // new[c] = old[rr_src(c)] over global slots; chunk boundaries move one value each way
                const T flr = __shfl_up_sync(kFull, vr[W - 2], 8);
                const T fli = __shfl_up_sync(kFull, vi[W - 2], 8);
                const T frr = __shfl_down_sync(kFull, vr[1], 8);
                const T fri = __shfl_down_sync(kFull, vi[1], 8);
                T nr[W], ni[W];
                nr[0] = chunk == 0 ? vr[0] : flr;
                ni[0] = chunk == 0 ? vi[0] : fli;
                nr[2] = chunk == 0 ? vr[1] : vr[0];
                ni[2] = chunk == 0 ? vi[1] : vi[0];
#pragma unroll
                for (int e = 4; e < W; e += 2) { nr[e] = vr[e - 2]; ni[e] = vi[e - 2]; }
#pragma unroll
                for (int o = 1; o <= W - 3; o += 2) { nr[o] = vr[o + 2]; ni[o] = vi[o + 2]; }
                nr[W - 1] = chunk == CH - 1 ? vr[W - 2] : frr;
                ni[W - 1] = chunk == CH - 1 ? vi[W - 2] : fri;
#pragma unroll
                for (int e = 0; e < W; ++e) { vr[e] = nr[e]; vi[e] = ni[e]; }
            }
            __syncthreads();
            int* tmp = ix; ix = ixn; ixn = tmp;
        }
    }
    return sweeps;
}

// theta entries (i <= j) into the packed triangle: h_e - sum_children 1 (x) m + sum_parents m,
// m = (1 - th) nu + th zeta (zeta == nullptr: m = nu).  FP64 path reads h64.
template <int D, typename T, typename Acc>
__device__ void assemble_packed(const DevProblem& P, const RegionInfo& R, int inst, Acc A,
                                const float2* __restrict__ nu, const float2* __restrict__ zeta, float th, bool use_h64) {
    constexpr int NT = CtaCfg<D>::NT;
    const int64_t mbase = (int64_t)inst * P.msg_elems;
    const float om = 1.0f - th;
    for (int e = threadIdx.x; e < D * D; e += NT) {
        const int i = e / D, j = e % D;
        if (i > j) continue;
        T re = T(0), im = T(0);
        if (R.h_off >= 0) {
            if (use_h64) {
                const double2 v = P.h64[(int64_t)inst * P.h_elems + R.h_off + e];
                re = T(v.x); im = T(v.y);
            } else {
                const float2 v = P.h32[(int64_t)inst * P.h_elems + R.h_off + e];
                re = T(v.x); im = T(v.y);
            }
        }
        for (int q = R.child_begin; q < R.child_end; ++q) {
            const PairInfo pi = P.child_info[q];
            if (((i ^ j) & ~pi.mask) != 0) continue;
            const int Df = 1 << pi.kf;
            const int64_t o = mbase + pi.off + (int64_t)pext8(i, pi.mask) * Df + pext8(j, pi.mask);
            float2 m = nu[o];
            if (zeta) { const float2 z = zeta[o]; m.x = om * m.x + th * z.x; m.y = om * m.y + th * z.y; }
            re -= T(m.x); im -= T(m.y);
        }
        for (int q = R.parent_begin; q < R.parent_end; ++q) {
            const PairInfo pi = P.parent_info[q];
            const int64_t o = mbase + pi.off + e;
            float2 m = nu[o];
            if (zeta) { const float2 z = zeta[o]; m.x = om * m.x + th * z.x; m.y = om * m.y + th * z.y; }
            re += T(m.x); im += T(m.y);
        }
        if (i == j) im = T(0);
        typename V2<T>::t v; v.x = re; v.y = im;
        A.set(A.sig(i), A.sig(j), v);
    }
}

// FP32 pass version: message entries from pass_entry (pending Alg. 2 update applied); the
// region owns its parent messages and also stores their conjugate (lower-triangle) entries.
template <int D, typename Acc>
__device__ void assemble_packed_io(const DevProblem& P, const RegionInfo& R, int inst, Acc A, const PassIO& io,
                                   const dev::Thetas& T) {
    constexpr int NT = CtaCfg<D>::NT;
    const int64_t mbase = (int64_t)inst * P.msg_elems;
    const int64_t rbase = (int64_t)inst * P.rho_elems;
    const bool owner_writes = io.zeta_in && io.pending;
    for (int e = threadIdx.x; e < D * D; e += NT) {
        const int i = e / D, j = e % D;
        if (i > j) continue;
        float re = 0.f, im = 0.f;
        if (R.h_off >= 0) {
            const float2 v = P.h32[(int64_t)inst * P.h_elems + R.h_off + e];
            re = v.x; im = v.y;
        }
        for (int q = R.child_begin; q < R.child_end; ++q) {
            const PairInfo pi = P.child_info[q];
            if (((i ^ j) & ~pi.mask) != 0) continue;
            const int Df = 1 << pi.kf;
            const int64_t x = (int64_t)pext8(i, pi.mask) * Df + pext8(j, pi.mask);
            const float2 m = dev::pass_entry(io, T, mbase + pi.off + x, rbase + pi.child_rho + x, false);
            re -= m.x; im -= m.y;
        }
        for (int q = R.parent_begin; q < R.parent_end; ++q) {
            const PairInfo pi = P.parent_info[q];
            float2 n, z;
            const float2 m = dev::pass_entry(io, T, mbase + pi.off + e, rbase + R.rho_off + e, true, &n, &z);
            if (owner_writes && i < j) {
                const int64_t et = mbase + pi.off + (int64_t)j * D + i;
                io.nu_out[et] = make_float2(n.x, -n.y);
                io.zeta_out[et] = make_float2(z.x, -z.y);
            }
            re += m.x; im += m.y;
        }
        if (i == j) im = 0.f;
        A.set(A.sig(i), A.sig(j), make_float2(re, im));
    }
}

// off-diagonal block pairs (k < l) in row order
template <int D, typename T>
__device__ void build_table(unsigned short* tab) {
    constexpr int n = D / 2;
    const int t = threadIdx.x;
    if (t < n) {
        const int off = t * (n - 1) - ((t * (t - 1)) >> 1);
        for (int l = t + 1; l < n; ++l) tab[off + (l - t - 1)] = (unsigned short)((t << 8) | l);
    }
}


// ---------------------------------------------------------------------------------------------
// Tensor-core back-transform for the FP32 CTA pass (D = 128): rho = W W^dagger with
// W = V diag(sqrt p), as one real GEMM  [rho_r; rho_i] = A B^T  with
//   A = [[W_r, W_i], [W_i, -W_r]]  (2D x 2D),   B = [W_r, W_i]  (D x 2D, = the first D rows of A),
// on tcgen05.mma kind::tf32 with FP32 accumulators in tensor memory.  FP32 accuracy from three
// TF32 products per term (x = hi + lo, hi = x with the low 13 mantissa bits cleared, lo = x - hi
// exact; A B^T ~ A_hi B_hi + A_hi B_lo + A_lo B_hi, the dropped lo*lo term is below 2^-21
// relative).  K = 2D is staged in chunks of KC columns (KC / 2 values of c, real then imaginary
// part; KC = 32) into two alternating shared-memory buffers while the previous chunk's MMAs run.
// Operands use the K-major layout without swizzle: core matrices of 8 rows x 16 bytes, K-adjacent
// core matrices 128 bytes apart (leading byte offset), 8-row groups KC * 32 bytes apart (stride
// byte offset).  One elected thread issues the MMAs and commits them to an mbarrier; all waits
// are bounded and report DEV_ERR_TIMEOUT.
// ---------------------------------------------------------------------------------------------
namespace tc {

// K columns per chunk
template <int D> struct TcKC { static constexpr int v = 32; };
constexpr uint32_t kLBO = 128;         // bytes between K-adjacent core matrices
template <int KC> struct TcSBO { static constexpr uint32_t v = (KC / 4) * 128; };   // bytes between 8-row groups
constexpr unsigned long long kWaitNs = 500000000ull;

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// instruction descriptor of kind::tf32: F32 accumulator, TF32 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// shared-memory matrix descriptor: start address, leading / stride byte offsets, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
                 :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}

__device__ __forceinline__ void commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mbar) : "memory");
}

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded wait for the phase with the given parity; false after kWaitNs
__device__ __forceinline__ bool wait_parity(uint32_t mbar, uint32_t parity) {
    const unsigned long long t0 = now_ns();
    for (;;) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n" : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
        if (now_ns() - t0 > kWaitNs) return false;
    }
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// byte offset of element (row m, K column kk) of one operand buffer
template <int KC>
__device__ __forceinline__ uint32_t off(int m, int kk) {
    return (uint32_t)((m >> 3) * TcSBO<KC>::v + (kk >> 2) * kLBO + (m & 7) * 16 + (kk & 3) * 4);
}

// 32 consecutive TMEM columns of this warp's 32 lanes
__device__ __forceinline__ void ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                 "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                   "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr) : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Stage K chunk j (c in [16 j, 16 j + 16)) of A = [[W_r, W_i], [W_i, -W_r]] as hi and lo parts.
// The thread holding row `row`, columns [vc W, vc W + W) of V writes when the chunk is in them;
// OFF is the chunk's first column inside the thread's W columns (compile-time).
template <int D, int OFF>
__device__ __forceinline__ void stage_rows(unsigned char* hi, unsigned char* lo, int row, const float* q,
                                           const float (&vr)[D / 4], const float (&vi)[D / 4], int c0) {
    constexpr int KC = TcKC<D>::v;
#pragma unroll
    for (int g = 0; g < KC / 8; ++g) {   // K groups of 4: real parts of c0 + 4g .. c0 + 4g + 3
        float wr[4], wi[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float s = q[c0 + 4 * g + e];
            wr[e] = vr[OFF + 4 * g + e] * s;
            wi[e] = vi[OFF + 4 * g + e] * s;
        }
        // row: [W_r | W_i]; row + D: [W_i | -W_r]
        const float4 a0 = make_float4(wr[0], wr[1], wr[2], wr[3]);
        const float4 a1 = make_float4(wi[0], wi[1], wi[2], wi[3]);
        const float4 b0 = a1;
        const float4 b1 = make_float4(-wr[0], -wr[1], -wr[2], -wr[3]);
        const float4 parts[4] = {a0, a1, b0, b1};
        const int rows[4] = {row, row, row + D, row + D};
        const int cols[4] = {4 * g, KC / 2 + 4 * g, 4 * g, KC / 2 + 4 * g};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float4 x = parts[u];
            const float4 h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
            const float4 l = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
            const uint32_t o = off<KC>(rows[u], cols[u]);
            *reinterpret_cast<float4*>(hi + o) = h;
            *reinterpret_cast<float4*>(lo + o) = l;
        }
    }
}

}  // namespace tc

// rho = W W^dagger on the tensor cores into two padded planes Rr, Ri (D x (D+1) floats each, the
// upper triangle of rho is read from them).  Returns false if a wait timed out (DEV_ERR_TIMEOUT).
template <int D>
__device__ bool backtransform_tc(const DevProblem& P, unsigned char* sm, float* pw, uint64_t* mbar, uint32_t* tslot,
                                 const float (&vr)[D / 4], const float (&vi)[D / 4], int row, int chunk) {
    using S = CtaSmem<D, float>;
    constexpr int W = D / 4;
    constexpr int M = 128;                    // MMA rows per tile
    constexpr int MT = (2 * D) / M;           // A tiles: 1 (D = 64) or 2 (D = 128)
    constexpr int KC = tc::TcKC<D>::v;
    constexpr uint32_t SBO = tc::TcSBO<KC>::v;
    constexpr int NCH = (2 * D) / KC;         // K chunks
    constexpr uint32_t NCOL = D == 64 ? 64u : 256u;   // TMEM columns (power of two >= 32)
    constexpr uint32_t PART = (uint32_t)(2 * D) * KC * 4;   // bytes of one operand part (2D rows x KC)
    static_assert(4 * PART <= S::buf_bytes, "tensor-core operands do not fit the buffer");
    const int t = threadIdx.x, warp = t >> 5;
    const uint32_t base = tc::saddr(sm);
    const uint32_t mb0 = tc::saddr(mbar), mb1 = tc::saddr(mbar + 1);
    const uint32_t idesc = tc::idesc_tf32(M, D);
    bool ok = true;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(tc::saddr(tslot)), "r"(NCOL) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mb0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mb1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    int last = -1;   // last chunk whose MMAs were issued and committed
    for (int j = 0; j < NCH; ++j) {
        const int b = j & 1;
        unsigned char* hi = sm + (size_t)(2 * b) * PART;
        unsigned char* lo = hi + PART;
        // the buffer is free once the MMAs of chunk j - 2 have completed; after a timed-out wait
        // (any thread) nothing more is staged or issued
        const bool late = j >= 2 && !tc::wait_parity(b ? mb1 : mb0, (uint32_t)((j / 2 - 1) & 1));
        if (__syncthreads_or(late)) { ok = false; break; }
        const int c0 = KC / 2 * j;            // first c of the chunk
        if (chunk == c0 / W) {   // the chunk's KC / 2 columns start at 0 or at W / 2 of the thread's W
            if (c0 % W == 0) tc::stage_rows<D, 0>(hi, lo, row, pw, vr, vi, c0);
            else tc::stage_rows<D, W / 2>(hi, lo, row, pw, vr, vi, c0);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ahi = base + (uint32_t)(2 * b) * PART, alo = ahi + PART;
#pragma unroll
            for (int s = 0; s < KC / 8; ++s) {
                const uint32_t ko = (uint32_t)(2 * s) * tc::kLBO;   // 8 K columns = 2 core matrices
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) {
                    const uint32_t mo = (uint32_t)mt * (M / 8) * SBO;
                    const uint32_t d = tmem + (uint32_t)(mt * D);
                    const uint32_t acc0 = (j > 0 || s > 0) ? 1u : 0u;
                    tc::mma(d, tc::sdesc(ahi + mo + ko, tc::kLBO, SBO), tc::sdesc(ahi + ko, tc::kLBO, SBO), idesc, acc0);
                    tc::mma(d, tc::sdesc(ahi + mo + ko, tc::kLBO, SBO), tc::sdesc(alo + ko, tc::kLBO, SBO), idesc, 1u);
                    tc::mma(d, tc::sdesc(alo + mo + ko, tc::kLBO, SBO), tc::sdesc(ahi + ko, tc::kLBO, SBO), idesc, 1u);
                }
            }
            tc::commit(b ? mb1 : mb0);
        }
        last = j;
    }
    // the last commit covers every MMA issued before it: wait for it (bounded) before the
    // accumulators are read and the tensor memory is released
    if (last >= 0 && !tc::wait_parity((last & 1) ? mb1 : mb0, (uint32_t)((last / 2) & 1))) ok = false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // accumulators -> padded planes (the operand buffers are free now)
    float* Rr = reinterpret_cast<float*>(sm);
    float* Ri = Rr + D * (D + 1);
    {
        const int q = warp & 3, g = warp >> 2, lane = t & 31;
        float v[32];
        if constexpr (D == 128) {
            const int i = 32 * q + lane;
            tc::ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * g), v);
#pragma unroll
            for (int e = 0; e < 32; ++e) Rr[i * (D + 1) + 32 * g + e] = v[e];
            tc::ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(D + 32 * g), v);
#pragma unroll
            for (int e = 0; e < 32; ++e) Ri[i * (D + 1) + 32 * g + e] = v[e];
        } else {
            const int lanei = 32 * q + lane;
            tc::ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * g), v);
            float* dst = lanei < D ? Rr + lanei * (D + 1) : Ri + (lanei - D) * (D + 1);
#pragma unroll
            for (int e = 0; e < 32; ++e) dst[32 * g + e] = v[e];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(NCOL) : "memory");
    }
    if (!ok && t == 0) atomicOr(P.err, DEV_ERR_TIMEOUT);
    return ok;
}

// Warm start of a CTA region's eigensolve (D = 64, 128) from the basis V its previous pass stored
// at Vg (D x D row-major complex: natural rows, eigenvector labels as columns), in two parts
// around the assembly of theta (which needs the shared buffer `buf`, D x (D + 1) complex):
//   warm_cta_basis: one Newton-Schulz step, V <- V (3 I - V^H V) / 2 (V^H V formed from V staged
//     in buf, then held in buf while each thread forms its rows' chunk of the new V from V's row
//     in global memory), written back to Vg;
//   warm_cta_rotate (after the assembly): T = theta V (theta from buf, V from Vg) into buf, then
//     V^H T (V from Vg, T from buf) into buf at the Jacobi's positions (sig), upper triangle.
// Both products run over the TR x TC register tiles of the rho formation.  CTA barriers inside.
template <int D>
struct WarmTile {
    static constexpr int NT = CtaCfg<D>::NT, TR = CtaCfg<D>::TR, TC = CtaCfg<D>::TC, CS = D / TC;
    float r[TR][TC], i[TR][TC];
    int i0, cb;
    __device__ __forceinline__ WarmTile() {
        const int t = threadIdx.x;
        i0 = (t / CS) * TR;
        cb = t % CS;
#pragma unroll
        for (int a = 0; a < TR; ++a)
#pragma unroll
            for (int b = 0; b < TC; ++b) { r[a][b] = 0.f; i[a][b] = 0.f; }
    }
    // += conj(x[a]) * y[b]  (cx) or x[a] * y[b]
    template <bool CX>
    __device__ __forceinline__ void mac(const float2 (&x)[TR], const float2 (&y)[TC]) {
#pragma unroll
        for (int a = 0; a < TR; ++a)
#pragma unroll
            for (int b = 0; b < TC; ++b) {
                if (CX) {
                    r[a][b] = fmaf(x[a].x, y[b].x, fmaf(x[a].y, y[b].y, r[a][b]));
                    i[a][b] = fmaf(x[a].x, y[b].y, fmaf(-x[a].y, y[b].x, i[a][b]));
                } else {
                    r[a][b] = fmaf(x[a].x, y[b].x, fmaf(-x[a].y, y[b].y, r[a][b]));
                    i[a][b] = fmaf(x[a].x, y[b].y, fmaf(x[a].y, y[b].x, i[a][b]));
                }
            }
    }
    // the tile into a plain D x D row-major array
    __device__ __forceinline__ void store(float2* out) const {
#pragma unroll
        for (int a = 0; a < TR; ++a)
#pragma unroll
            for (int b = 0; b < TC; ++b) out[(i0 + a) * D + cb + CS * b] = make_float2(r[a][b], i[a][b]);
    }
};

template <int D>
__device__ void warm_cta_basis(float2* buf, float2* Vg) {
    using WT = WarmTile<D>;
    constexpr int NT = WT::NT, TR = WT::TR, TC = WT::TC, CS = WT::CS, W = D / 4;
    const int t = threadIdx.x;
    {   // V into buf (float4 copies: D x D complex)
        const float4* src = reinterpret_cast<const float4*>(Vg);
        float4* dst = reinterpret_cast<float4*>(buf);
        for (int e = t; e < D * D / 2; e += NT) dst[e] = src[e];
    }
    __syncthreads();
    WT G;   // G = V^H V: G[i][c] = sum_k conj(V[k][i]) V[k][c]
    for (int k = 0; k < D; ++k) {
        const float2* vk = buf + k * D;
        float2 x[TR], y[TC];
#pragma unroll
        for (int a = 0; a < TR; ++a) x[a] = vk[G.i0 + a];
#pragma unroll
        for (int b = 0; b < TC; ++b) y[b] = vk[G.cb + CS * b];
        G.template mac<true>(x, y);
    }
    __syncthreads();
    G.store(buf);
    __syncthreads();
    // rows' chunk of V (3 I - G) / 2: thread (row, chunk) forms V'[row][chunk W + m]
    const int row = vrow_of(t), chunk = vchunk_of(t);
    float ur[W], ui[W];
#pragma unroll
    for (int m = 0; m < W; ++m) { ur[m] = 0.f; ui[m] = 0.f; }
    const float2* vrow = Vg + (int64_t)row * D;
    for (int c = 0; c < D; ++c) {
        const float2 a = vrow[c];
        const float2* gc = buf + c * D + chunk * W;
#pragma unroll
        for (int m = 0; m < W; ++m) {
            const float2 g = gc[m];
            ur[m] = fmaf(a.x, g.x, fmaf(-a.y, g.y, ur[m]));
            ui[m] = fmaf(a.x, g.y, fmaf(a.y, g.x, ui[m]));
        }
    }
    __syncthreads();   // every thread has read V's rows from Vg (its own chunk is written by it alone)
#pragma unroll
    for (int m = 0; m < W; ++m) {
        float2* e = Vg + (int64_t)row * D + chunk * W + m;
        const float2 o = *e;
        *e = make_float2(fmaf(1.5f, o.x, -0.5f * ur[m]), fmaf(1.5f, o.y, -0.5f * ui[m]));
    }
    __syncthreads();
}

template <int D>
__device__ void warm_cta_rotate(float2* buf, const float2* Vg) {
    using WT = WarmTile<D>;
    constexpr int TR = WT::TR, TC = WT::TC, CS = WT::CS;
    Full<float> A{buf, D};
    WT T;   // T = theta V: T[i][c] = sum_k theta[i][k] V[k][c]
    int si[TR];
#pragma unroll
    for (int a = 0; a < TR; ++a) si[a] = A.sig(T.i0 + a);
    for (int k = 0; k < D; ++k) {
        const int sk = A.sig(k);
        const float2* vk = Vg + (int64_t)k * D;
        float2 x[TR], y[TC];
#pragma unroll
        for (int a = 0; a < TR; ++a) x[a] = A.get(si[a], sk);
#pragma unroll
        for (int b = 0; b < TC; ++b) y[b] = vk[T.cb + CS * b];
        T.template mac<false>(x, y);
    }
    __syncthreads();
    T.store(buf);
    __syncthreads();
    WT M;   // V^H T: M[i][c] = sum_k conj(V[k][i]) T[k][c]
    for (int k = 0; k < D; ++k) {
        const float2* vk = Vg + (int64_t)k * D;
        const float2* tk = buf + k * D;
        float2 x[TR], y[TC];
#pragma unroll
        for (int a = 0; a < TR; ++a) x[a] = vk[M.i0 + a];
#pragma unroll
        for (int b = 0; b < TC; ++b) y[b] = tk[M.cb + CS * b];
        M.template mac<true>(x, y);
    }
    __syncthreads();
    // upper triangle at the Jacobi's positions (exactly Hermitian, real diagonal)
#pragma unroll
    for (int a = 0; a < TR; ++a)
#pragma unroll
        for (int b = 0; b < TC; ++b) {
            const int ii = M.i0 + a, jj = M.cb + CS * b;
            if (ii < jj) A.set(A.sig(ii), A.sig(jj), make_float2(M.r[a][b], M.i[a][b]));
            else if (ii == jj) A.set(A.sig(ii), A.sig(ii), make_float2(M.r[a][b], 0.f));
        }
    __syncthreads();
}

template <int D>
__global__ void __launch_bounds__(CtaCfg<D>::NT) region_pass_cta_kernel(const DevProblem P, const PassIO io,
                                                                        const int32_t* __restrict__ cls,
                                                                        const int32_t count, const int k) {
    using S = CtaSmem<D, float>;
    constexpr int NT = CtaCfg<D>::NT;
    constexpr int W = D / 4;
    constexpr int TR = CtaCfg<D>::TR, TC = CtaCfg<D>::TC;
    extern __shared__ __align__(16) unsigned char sm[];
    float2* buf = reinterpret_cast<float2*>(sm);
    RotC<float>* prm = reinterpret_cast<RotC<float>*>(sm + S::off_prm);
    int* idx0 = reinterpret_cast<int*>(sm + S::off_idx);
    int* idx1 = idx0 + D;
    unsigned short* tab = reinterpret_cast<unsigned short*>(sm + S::off_tab);
    float* lam = reinterpret_cast<float*>(sm + S::off_lam);
    float* pw = lam + D;
    float* red = reinterpret_cast<float*>(sm + S::off_red);
    const int t = threadIdx.x;
    const int inst = blockIdx.x / count;
    const int r = cls[blockIdx.x % count];
    const RegionInfo R = P.reg[r];
    const bool nest = P.st->variant == 1;
    const dev::Thetas Th = dev::pass_thetas(P, io);
    if (io.writer && blockIdx.x == 0 && t == 0) dev::advance_theta(P, io);
    build_table<D, float>(tab);
    Full<float> A{buf, D};
    if (t < D) idx0[t] = A.sig(t);
    // warm start from the stored basis (uniform over the CTA)
    const bool warm = P.warm != nullptr && P.warm_off[k] >= 0 && !P.st->cold;
    float2* Vg = warm ? P.warm + P.warm_off[k] + (int64_t)blockIdx.x * (D * D) : nullptr;
    if (warm) warm_cta_basis<D>(buf, Vg);
    assemble_packed_io<D>(P, R, inst, A, io, Th);
    __syncthreads();
    if (warm) warm_cta_rotate<D>(buf, Vg);
    const int row = vrow_of(t), chunk = vchunk_of(t);
    float vr[W], vi[W];
    if (warm) {
#pragma unroll
        for (int m = 0; m < W; ++m) {
            const float2 v = Vg[(int64_t)row * D + chunk * W + m];
            vr[m] = v.x; vi[m] = v.y;
        }
    } else {
#pragma unroll
        for (int m = 0; m < W; ++m) { vr[m] = (chunk * W + m == row) ? 1.f : 0.f; vi[m] = 0.f; }
    }
    float norm2, off2;
    const int sweeps =
        jacobi_cta<D, float, true>(A, prm, idx0, idx1, tab, red, vr, vi, P.st->max_sweeps, 1e-12f, norm2, off2);
    if (warm) {   // the eigenvectors as the next pass's starting basis (the identity if not finite)
        bool fin = true;
#pragma unroll
        for (int m = 0; m < W; ++m) fin = fin && isfinite(vr[m]) && isfinite(vi[m]);
        const bool bad = __syncthreads_or(fin ? 0 : 1) != 0;
#pragma unroll
        for (int m = 0; m < W; ++m)
            Vg[(int64_t)row * D + chunk * W + m] = bad ? make_float2(chunk * W + m == row ? 1.f : 0.f, 0.f)
                                                       : make_float2(vr[m], vi[m]);
    }
    // the slot maps are back to the identity after whole sweeps: diag = eigenvalues
    if (t < D) lam[t] = A.dget(A.sig(t)).x;
    __syncthreads();
    float lmin = lam[0];
    for (int i = 1; i < D; ++i) lmin = fminf(lmin, lam[i]);
    float F, Z = 0.f;
    if (nest) {
        const float beta = (float)P.st->beta;
        for (int i = 0; i < D; ++i) Z += expf(-beta * (lam[i] - lmin));
        F = lmin - logf(Z) / beta;
        if (t < D) pw[t] = sqrtf(expf(-beta * (lam[t] - lmin)) / Z);
    } else {
        const float tau = (float)P.st->degen_tol * fmaxf(1.0f, sqrtf(norm2));
        for (int i = 0; i < D; ++i) Z += (lam[i] - lmin <= tau) ? 1.f : 0.f;
        F = lmin;
        if (t < D) pw[t] = (lam[t] - lmin <= tau) ? sqrtf(1.0f / Z) : 0.f;
    }
    __syncthreads();
    // the tensor-core back-transform is built for D = 128 only: at D = 64 a kernel containing it
    // ran with half the resident CTAs per SM (one instead of two) and was slower overall
    bool use_tc = false;
    if constexpr (D == 128) use_tc = ((P.tc_backtransform >> (k - 6)) & 1) != 0;
    if (use_tc) {
        if constexpr (D == 128) {
            uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + S::off_mbar);
            uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S::off_mbar + 16);
            backtransform_tc<D>(P, sm, pw, mbar, tslot, vr, vi, row, chunk);
            // rho from the planes: upper triangle as computed, lower = its conjugate, real diagonal
            const float* Rr = reinterpret_cast<const float*>(sm);
            const float* Ri = Rr + D * (D + 1);
            auto rho_at = [&](int i, int j) -> float2 {
                if (i < j) return make_float2(Rr[i * (D + 1) + j], Ri[i * (D + 1) + j]);
                if (i > j) return make_float2(Rr[j * (D + 1) + i], -Ri[j * (D + 1) + i]);
                return make_float2(Rr[i * (D + 1) + i], 0.f);
            };
            if (R.rho_off >= 0) {
                float2* dst = io.rho_out + (int64_t)inst * P.rho_elems + R.rho_off;
                for (int e = t; e < D * D; e += NT) dst[e] = rho_at(e / D, e % D);
            }
            float2* trb = io.tr_out + (int64_t)inst * P.msg_elems;
            for (int q = R.child_begin; q < R.child_end; ++q) {
                const PairInfo pi = P.child_info[q];
                const int M = pi.mask, Mc = (D - 1) & ~M, kf = pi.kf, Df = 1 << kf, nrest = D >> kf;
                for (int o = t; o < Df * Df; o += NT) {
                    const int ra = pdep8(o >> kf, M), rbb = pdep8(o & (Df - 1), M);
                    float sr = 0.f, si = 0.f;
                    for (int c = 0; c < nrest; ++c) {
                        const int x = pdep8(c, Mc);
                        const float2 v = rho_at(ra | x, rbb | x);
                        sr += v.x; si += v.y;
                    }
                    trb[pi.off + o] = make_float2(sr, si);
                }
            }
        }
    } else {
        // W^T[c][row] = V[row][c] sqrt(p_c)   (overwrites the triangle, no longer needed)
#pragma unroll
        for (int m = 0; m < W; ++m) {
            const int c = chunk * W + m;
            const float q = pw[c];
            buf[c * D + row] = make_float2(vr[m] * q, vi[m] * q);
        }
        __syncthreads();
        // rho = W W^dagger in TR x TC register tiles: rho[i][c] = sum_k W[i][k] conj(W[c][k]); a thread
        // owns rows i0 .. i0+TR-1 and the strided columns cb + (D/TC) b, so that consecutive threads
        // read and write consecutive columns (no shared-memory bank conflicts)
        const int rb = t / (D / TC), cb = t % (D / TC);
        const int i0 = rb * TR;
        constexpr int CS = D / TC;
        float accr[TR][TC], acci[TR][TC];
#pragma unroll
        for (int a = 0; a < TR; ++a)
#pragma unroll
            for (int b = 0; b < TC; ++b) { accr[a][b] = 0.f; acci[a][b] = 0.f; }
        for (int kk = 0; kk < D; ++kk) {
            const float2* wk = buf + kk * D;
            float2 wi[TR], wc[TC];
#pragma unroll
            for (int a = 0; a < TR; ++a) wi[a] = wk[i0 + a];
#pragma unroll
            for (int b = 0; b < TC; ++b) wc[b] = wk[cb + CS * b];
#pragma unroll
            for (int a = 0; a < TR; ++a)
#pragma unroll
                for (int b = 0; b < TC; ++b) {
                    accr[a][b] += wi[a].x * wc[b].x + wi[a].y * wc[b].y;
                    acci[a][b] += wi[a].y * wc[b].x - wi[a].x * wc[b].y;
                }
        }
        __syncthreads();
#pragma unroll
        for (int a = 0; a < TR; ++a)
#pragma unroll
            for (int b = 0; b < TC; ++b) buf[(i0 + a) * D + cb + CS * b] = make_float2(accr[a][b], acci[a][b]);
        __syncthreads();
        // exact Hermitian symmetry: lower triangle := conj(upper), real diagonal
        for (int e = t; e < D * D; e += NT) {
            const int i = e / D, j = e % D;
            if (i > j) { const float2 u = buf[j * D + i]; buf[e] = make_float2(u.x, -u.y); }
            else if (i == j) buf[e].y = 0.f;
        }
        __syncthreads();
        if (R.rho_off >= 0) {
            float4* dst = reinterpret_cast<float4*>(io.rho_out + (int64_t)inst * P.rho_elems + R.rho_off);
            const float4* srcv = reinterpret_cast<const float4*>(buf);
            for (int e = t; e < D * D / 2; e += NT) dst[e] = srcv[e];
        }
        float2* trb = io.tr_out + (int64_t)inst * P.msg_elems;
        for (int q = R.child_begin; q < R.child_end; ++q) {
            const PairInfo pi = P.child_info[q];
            const int M = pi.mask, Mc = (D - 1) & ~M, kf = pi.kf, Df = 1 << kf, nrest = D >> kf;
            for (int o = t; o < Df * Df; o += NT) {
                const int ra = pdep8(o >> kf, M), rbb = pdep8(o & (Df - 1), M);
                float sr = 0.f, si = 0.f;
                for (int c = 0; c < nrest; ++c) {
                    const int x = pdep8(c, Mc);
                    const float2 v = buf[(ra | x) * D + (rbb | x)];
                    sr += v.x; si += v.y;
                }
                trb[pi.off + o] = make_float2(sr, si);
            }
        }
    }
    if (t == 0) {
        P.val[(int64_t)inst * P.n_regions + r] = (double)F;
        if (!isfinite(F)) atomicOr(P.err, DEV_ERR_NUMERIC);
        atomicAdd(&P.sweeps[k], (unsigned long long)sweeps);
        if (off2 > 1e-12f * norm2) atomicAdd(&P.capped[k], 1ull);
    }
}

template <int D>
__global__ void __launch_bounds__(CtaCfg<D>::NT) certify_cta_kernel(const DevProblem P, const int32_t* __restrict__ cls,
                                                                    const int32_t count, const float2* __restrict__ msg) {
    using S = CtaSmem<D, double>;
    constexpr int W = D / 4;
    extern __shared__ __align__(16) unsigned char sm[];
    double2* buf = reinterpret_cast<double2*>(sm);
    RotC<double>* prm = reinterpret_cast<RotC<double>*>(sm + S::off_prm);
    int* idx0 = reinterpret_cast<int*>(sm + S::off_idx);
    int* idx1 = idx0 + D;
    unsigned short* tab = reinterpret_cast<unsigned short*>(sm + S::off_tab);
    double* red = reinterpret_cast<double*>(sm + S::off_red);
    const int t = threadIdx.x;
    const int inst = blockIdx.x / count;
    const int r = cls[blockIdx.x % count];
    const RegionInfo R = P.reg[r];
    build_table<D, double>(tab);
    Packed<double> A{buf, D};
    if (t < D) idx0[t] = A.sig(t);
    assemble_packed<D, double>(P, R, inst, A, msg, nullptr, 0.0f, true);
    __syncthreads();
    double vr[W], vi[W];
    double norm2, off2;
    jacobi_cta<D, double, false>(A, prm, idx0, idx1, tab, red, vr, vi, P.st->cert_sweeps, 1e-28, norm2, off2);
    double lmin = buf[0].x;
    for (int i = 1; i < D; ++i) lmin = fmin(lmin, buf[tri(i, i, D)].x);
    // Weyl: lambda_min >= min_i a_ii - ||offdiag||_F, a lower bound also when the cap stopped it
    lmin -= sqrt(off2);
    if (t == 0) {
        P.val64[(int64_t)inst * P.n_regions + r] = lmin;
        if (!isfinite(lmin)) atomicOr(P.err, DEV_ERR_NUMERIC);
        if (off2 > 1e-28 * norm2) atomicOr(P.err, DEV_ERR_NOCONV);
    }
}

// ---------------------------------------------------------------------------------------------
// D = 256 (regions of 8 sites).  theta's packed upper triangle (32,896 complex entries: 263 KB in
// FP32, 526 KB in FP64) and V (512 KB) exceed one SM's shared memory and registers.  The FP32
// Jacobi keeps theta in slot order in two packed triangles of this CTA's global scratch slot
// (L2-resident while the CTA runs), ping-ponged every round (jacobi256_slots); the FP64
// certification keeps the first part of its triangle in shared memory and the rest in the slot
// (Split accessor).  V is not carried through the sweeps: they append their rotations to a log in
// the slot (16 bytes per pair and round), and V is formed afterwards by replaying the log on 96
// rows at a time in shared memory: rows of V are independent (each is a row of the identity times
// J_1 J_2 ...), so each warp owns three rows and needs only a warp barrier between rounds.
// rho = W W^dagger (W = V diag(sqrt p)) is formed tile by tile into the slot and traced onto the
// children.  One 1024-thread CTA per SM, each looping over the regions of the launch.
constexpr int kBigD = 256;
constexpr int kBigN = kBigD / 2;
constexpr int kBigTri = kBigD * (kBigD + 1) / 2;   // 32,896 entries
constexpr int kBigNOFF = kBigN * (kBigN - 1) / 2;   // 8,128 off-diagonal 2x2 blocks
constexpr int kBigRB = 96;                          // V rows per batch (three per warp)
constexpr int kBigT = 64;                           // rho tile edge

struct BigSmem {
    static constexpr size_t prm_bytes = sizeof(RotC<double>) * (kBigN + 8);
    static constexpr size_t idx_bytes = sizeof(int) * 2 * kBigD;
    static constexpr size_t tab_bytes = (sizeof(unsigned short) * kBigNOFF + 15) / 16 * 16;
    static constexpr size_t lam_bytes = sizeof(double) * 2 * kBigD;
    static constexpr size_t red_bytes = sizeof(double) * 32;
    static constexpr size_t fixed = prm_bytes + idx_bytes + tab_bytes + lam_bytes + red_bytes;
    static constexpr size_t total = 227 * 1024;   // opt-in shared memory of one CTA
    static constexpr size_t tri_bytes = (total - fixed) / 16 * 16;
    static constexpr int ns64 = (int)(tri_bytes / sizeof(double2));
    static constexpr size_t off_prm = tri_bytes;
    static constexpr size_t off_idx = off_prm + prm_bytes;
    static constexpr size_t off_tab = off_idx + idx_bytes;
    static constexpr size_t off_lam = off_tab + tab_bytes;
    static constexpr size_t off_red = off_lam + lam_bytes;
    static constexpr size_t bytes = off_red + red_bytes;
    static_assert(bytes <= total, "D = 256 shared-memory layout");
    static_assert(sizeof(float2) * kBigRB * kBigD <= tri_bytes, "V batch");
    static_assert(sizeof(float2) * 2 * kBigT * (kBigT + 1) <= tri_bytes, "rho tiles");
};

// scratch slot (complex64 units): the two theta buffers of the FP32 Jacobi (packed upper
// triangles in slot order; the FP64 certification uses the same space for its overflow) | V (W
// after scaling) | rho | rotation log
constexpr int64_t kBigTriPad = ((int64_t)kBigTri + 1) / 2 * 2;
constexpr int64_t kBigOffV = 2 * kBigTriPad;
constexpr int64_t kBigOffR = kBigOffV + (int64_t)kBigD * kBigD;
constexpr int64_t kBigOffLog = kBigOffR + (int64_t)kBigD * kBigD;
static_assert(2 * (int64_t)(kBigTri - BigSmem::ns64) <= kBigOffLog, "FP64 overflow fits the slot");

__device__ __forceinline__ void rot_pair(float2& p, float2& q, const RotC<float>& R) {
    const float npr = R.c * p.x + (R.wr * q.x + R.wi * q.y);
    const float npi = R.c * p.y + (R.wr * q.y - R.wi * q.x);
    const float nqr = R.c * q.x - (R.wr * p.x - R.wi * p.y);
    const float nqi = R.c * q.y - (R.wr * p.y + R.wi * p.x);
    p = make_float2(npr, npi);
    q = make_float2(nqr, nqi);
}

// next slot of the entries in slot o (inverse of rr_src_c)
__host__ __device__ constexpr int rr_dst_c(int o, int D) {
    return o == 0 ? 0 : (o == 1 ? 2 : ((o & 1) ? o - 2 : (o == D - 2 ? D - 1 : o + 2)));
}

// Cyclic Jacobi of the D = 256 pass with theta in slot order, ping-ponged between two packed
// upper triangles in the CTA's global slot (L2-resident): a round reads every off-diagonal 2x2
// block (k, l) of the slot pairs (2k, 2k+1), (2l, 2l+1) at fixed addresses and writes each rotated
// entry at its next slots (rr_dst_c of its row and of its column; conjugated when that lands
// below the diagonal) in the other buffer; the diagonal block of pair k becomes exactly diagonal
// (the two entries of rot_params_d).  The rotations are those of jacobi_cta in the same order;
// the slot -> position map (which basis vector each slot holds) is tracked for the rotation log,
// from which V is formed afterwards.  After whole sweeps every entry is back in its own slot, so
// slot t's diagonal entry is the eigenvalue of V's column t.  Returns the sweeps run and the
// buffer holding the result.
__device__ int jacobi256_slots(float2* bufA, float2* bufB, RotC<float>* prm, int* idx0, int* idx1,
                               const unsigned short* tab, float* red, int max_sweeps, float tol2, float& norm2_out,
                               float& off_out, RotC<float>* log, float2*& result) {
    constexpr int D = kBigD, n = kBigN, NT = 1024, NOFF = kBigNOFF;
    const int t = threadIdx.x;
    float2* cur = bufA;
    float2* nxt = bufB;
    auto put = [&](float2* buf, int I, int J, float2 v) {
        const int a = rr_dst_c(I, D), b = rr_dst_c(J, D);
        if (a <= b) buf[tri(a, b, D)] = v;
        else buf[tri(b, a, D)] = make_float2(v.x, -v.y);
    };
    auto sums = [&](const float2* a, float& offd, float& dg) {
        offd = 0.f;
        dg = 0.f;
        for (int e = t; e < D * D; e += NT) {
            const int i = e / D, j = e % D;
            if (i < j) { const float2 v = a[tri(i, j, D)]; offd += v.x * v.x + v.y * v.y; }
        }
        for (int i = t; i < D; i += NT) { const float2 v = a[tri(i, i, D)]; dg += v.x * v.x + v.y * v.y; }
    };
    float up, dg;
    sums(cur, up, dg);
    const float norm2 = 2.f * block_sum<NT>(up, red) + block_sum<NT>(dg, red);
    norm2_out = norm2;
    const float thresh = tol2 * norm2;
    int* ix = idx0;
    int* ixn = idx1;
    int sweeps = 0;
    for (;;) {
        sums(cur, up, dg);
        const float off = 2.f * block_sum<NT>(up, red);
        off_out = off;
        if (off <= thresh || sweeps >= max_sweeps) break;
        ++sweeps;
        for (int r = 0; r < D - 1; ++r) {
            if (t < n) {
                const int p = 2 * t, q = 2 * t + 1;
                const float2 b = cur[tri(p, q, D)];
                float2 dnew;
                RotC<float> R;
                rot_params_d<float>(cur[tri(p, p, D)].x, cur[tri(q, q, D)].x, b.x, b.y, R, dnew);
                prm[t] = R;
                R.pad = __int_as_float(ix[p] | (ix[q] << 16));
                log[((size_t)(sweeps - 1) * (D - 1) + r) * n + t] = R;
                put(nxt, p, p, make_float2(dnew.x, 0.f));
                put(nxt, q, q, make_float2(dnew.y, 0.f));
                put(nxt, p, q, make_float2(0.f, 0.f));
            }
            __syncthreads();
            if (t < D) ixn[t] = ix[rr_src_c(t, D)];
            for (int v = t; v < NOFF; v += NT) {
                const int kl = tab[v];
                const int kk = kl >> 8, ll = kl & 255;
                const int i0 = 2 * kk, j0 = 2 * ll;
                const int r0 = tri(i0, j0, D), r1 = tri(i0 + 1, j0, D);
                float2 b00 = cur[r0], b01 = cur[r0 + 1], b10 = cur[r1], b11 = cur[r1 + 1];
                two_sided<float>(b00, b01, b10, b11, prm[kk], prm[ll]);
                put(nxt, i0, j0, b00);
                put(nxt, i0, j0 + 1, b01);
                put(nxt, i0 + 1, j0, b10);
                put(nxt, i0 + 1, j0 + 1, b11);
            }
            __syncthreads();
            float2* tb = cur; cur = nxt; nxt = tb;
            int* ti = ix; ix = ixn; ixn = ti;
        }
    }
    result = cur;
    return sweeps;
}

__global__ void __launch_bounds__(1024, 1) region_pass_cta256_kernel(const DevProblem P, const PassIO io,
                                                                     const int32_t* __restrict__ cls,
                                                                     const int32_t count, const int k) {
    using S = BigSmem;
    constexpr int D = kBigD, n = kBigN, NT = 1024;
    extern __shared__ __align__(16) unsigned char sm[];
    float2* tri_s = reinterpret_cast<float2*>(sm);
    RotC<float>* prm = reinterpret_cast<RotC<float>*>(sm + S::off_prm);
    int* idx0 = reinterpret_cast<int*>(sm + S::off_idx);
    int* idx1 = idx0 + D;
    unsigned short* tab = reinterpret_cast<unsigned short*>(sm + S::off_tab);
    float* lam = reinterpret_cast<float*>(sm + S::off_lam);
    float* pw = lam + D;
    float* red = reinterpret_cast<float*>(sm + S::off_red);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    float2* slot = P.big + (int64_t)blockIdx.x * P.big_slot;
    float2* Wg = slot + kBigOffV;
    float2* Rg = slot + kBigOffR;
    RotC<float>* logp = reinterpret_cast<RotC<float>*>(slot + kBigOffLog);
    const bool nest = P.st->variant == 1;
    const dev::Thetas Th = dev::pass_thetas(P, io);
    if (io.writer && blockIdx.x == 0 && t == 0) dev::advance_theta(P, io);
    build_table<D, float>(tab);
    const int max_sw = min(P.st->max_sweeps, P.big_log_sweeps);
    const int total = P.n_inst * count;
    for (int b = blockIdx.x; b < total; b += gridDim.x) {
        const int inst = b / count;
        const int r = cls[b % count];
        const RegionInfo R = P.reg[r];
        float2* thA = slot;
        float2* thB = slot + kBigTriPad;
        Split<float> A{tri_s, thA, 0, D};   // every entry in the slot's first buffer
        __syncthreads();   // the previous region's reads of shared memory and of the slot are done
        if (t < D) idx0[t] = t;
        assemble_packed_io<D>(P, R, inst, A, io, Th);
        __syncthreads();
        float norm2, off2;
        float2* th = thA;
        const int sweeps = jacobi256_slots(thA, thB, prm, idx0, idx1, tab, red, max_sw, 1e-12f, norm2, off2, logp, th);
        if (t < D) lam[t] = th[tri(t, t, D)].x;   // whole sweeps: slot t holds eigenvalue t
        __syncthreads();
        float lmin = lam[0];
        for (int i = 1; i < D; ++i) lmin = fminf(lmin, lam[i]);
        float F, Z = 0.f;
        if (nest) {
            const float beta = (float)P.st->beta;
            for (int i = 0; i < D; ++i) Z += expf(-beta * (lam[i] - lmin));
            F = lmin - logf(Z) / beta;
            if (t < D) pw[t] = sqrtf(expf(-beta * (lam[t] - lmin)) / Z);
        } else {
            const float tau = (float)P.st->degen_tol * fmaxf(1.0f, sqrtf(norm2));
            for (int i = 0; i < D; ++i) Z += (lam[i] - lmin <= tau) ? 1.f : 0.f;
            F = lmin;
            if (t < D) pw[t] = (lam[t] - lmin <= tau) ? sqrtf(1.0f / Z) : 0.f;
        }
        __syncthreads();
        // V from the log, kBigRB rows at a time (theta's shared part is free now); W = V diag(sqrt p)
        const int nrounds = sweeps * (D - 1);
        float2* Vs = tri_s;
        for (int row0 = 0; row0 < D; row0 += kBigRB) {
            const int rows = min(kBigRB, D - row0);
            for (int e = t; e < rows * D; e += NT) Vs[e] = make_float2((row0 + e / D == e % D) ? 1.f : 0.f, 0.f);
            __syncthreads();
            // warp w owns rows 3w .. 3w + 2 of the batch (those below `rows`)
            constexpr int RPW = kBigRB / 32;
            const int nr = max(0, min(RPW, rows - RPW * warp));
            float2* v0 = Vs + (RPW * warp) * D;
            // the next round's log records are loaded while this round's rotations run
            RotC<float> nxt[n / 32];
            if (nrounds > 0) {
#pragma unroll
                for (int m = 0; m < n / 32; ++m) nxt[m] = logp[lane + 32 * m];
            }
            for (int rd = 0; rd < nrounds; ++rd) {
                RotC<float> cur[n / 32];
#pragma unroll
                for (int m = 0; m < n / 32; ++m) cur[m] = nxt[m];
                if (rd + 1 < nrounds) {
                    const RotC<float>* lg = logp + (size_t)(rd + 1) * n;
#pragma unroll
                    for (int m = 0; m < n / 32; ++m) nxt[m] = lg[lane + 32 * m];
                }
#pragma unroll
                for (int m = 0; m < n / 32; ++m) {
                    const int pq = __float_as_int(cur[m].pad);
                    const int p = pq & 0xffff, q = pq >> 16;
#pragma unroll
                    for (int rr = 0; rr < RPW; ++rr)
                        if (rr < nr) rot_pair(v0[rr * D + p], v0[rr * D + q], cur[m]);
                }
                __syncwarp();
            }
            __syncthreads();
            for (int e = t; e < rows * D; e += NT) {
                const float2 v = Vs[e];
                const float q = pw[e % D];
                Wg[(int64_t)row0 * D + e] = make_float2(v.x * q, v.y * q);
            }
            __syncthreads();
        }
        // rho = W W^dagger, upper tiles (ti <= tj) of kBigT x kBigT: rho[i][j] = sum_c W[i][c] conj(W[j][c]);
        // thread (ty, tx) = (warp, lane) owns rows 2 ty, 2 ty + 1 and columns tx, tx + 32 of the tile
        {
            constexpr int T = kBigT, LD = T + 1;
            float2* Wa = tri_s;            // [T][LD]: rows of the tile's row block, c in the chunk
            float2* Wb = tri_s + T * LD;   // [T][LD]: transposed, Wb[c][j]
            for (int ti = 0; ti < D / T; ++ti)
                for (int tj = ti; tj < D / T; ++tj) {
                    float2 acc[2][2];
#pragma unroll
                    for (int a = 0; a < 2; ++a)
#pragma unroll
                        for (int bb = 0; bb < 2; ++bb) acc[a][bb] = make_float2(0.f, 0.f);
                    for (int c0 = 0; c0 < D; c0 += T) {
                        for (int e = t; e < T * T; e += NT) {
                            const int i = e / T, c = e % T;
                            Wa[i * LD + c] = Wg[(int64_t)(ti * T + i) * D + c0 + c];
                            Wb[c * LD + i] = Wg[(int64_t)(tj * T + i) * D + c0 + c];
                        }
                        __syncthreads();
                        for (int c = 0; c < T; ++c) {
                            const float2 a0 = Wa[(2 * warp) * LD + c], a1 = Wa[(2 * warp + 1) * LD + c];
                            const float2 b0 = Wb[c * LD + lane], b1 = Wb[c * LD + lane + 32];
                            const float2 av[2] = {a0, a1}, bv[2] = {b0, b1};
#pragma unroll
                            for (int a = 0; a < 2; ++a)
#pragma unroll
                                for (int bb = 0; bb < 2; ++bb) {
                                    acc[a][bb].x += av[a].x * bv[bb].x + av[a].y * bv[bb].y;
                                    acc[a][bb].y += av[a].y * bv[bb].x - av[a].x * bv[bb].y;
                                }
                        }
                        __syncthreads();
                    }
#pragma unroll
                    for (int a = 0; a < 2; ++a)
#pragma unroll
                        for (int bb = 0; bb < 2; ++bb)
                            Rg[(int64_t)(ti * T + 2 * warp + a) * D + tj * T + lane + 32 * bb] = acc[a][bb];
                }
        }
        __syncthreads();
        // exact Hermitian symmetry: lower triangle := conj(upper), real diagonal
        for (int e = t; e < D * D; e += NT) {
            const int i = e / D, j = e % D;
            if (i > j) { const float2 u = Rg[j * D + i]; Rg[e] = make_float2(u.x, -u.y); }
            else if (i == j) Rg[e].y = 0.f;
        }
        __syncthreads();
        if (R.rho_off >= 0) {
            float2* dst = io.rho_out + (int64_t)inst * P.rho_elems + R.rho_off;
            for (int e = t; e < D * D; e += NT) dst[e] = Rg[e];
        }
        float2* trb = io.tr_out + (int64_t)inst * P.msg_elems;
        for (int q = R.child_begin; q < R.child_end; ++q) {
            const PairInfo pi = P.child_info[q];
            const int M = pi.mask, Mc = (D - 1) & ~M, kf = pi.kf, Df = 1 << kf, nrest = D >> kf;
            for (int o = t; o < Df * Df; o += NT) {
                const int ra = pdep8(o >> kf, M), rbb = pdep8(o & (Df - 1), M);
                float sr = 0.f, si = 0.f;
                for (int c = 0; c < nrest; ++c) {
                    const int x = pdep8(c, Mc);
                    const float2 v = Rg[(ra | x) * D + (rbb | x)];
                    sr += v.x; si += v.y;
                }
                trb[pi.off + o] = make_float2(sr, si);
            }
        }
        if (t == 0) {
            P.val[(int64_t)inst * P.n_regions + r] = (double)F;
            if (!isfinite(F)) atomicOr(P.err, DEV_ERR_NUMERIC);
            atomicAdd(&P.sweeps[k], (unsigned long long)sweeps);
            if (off2 > 1e-12f * norm2) atomicAdd(&P.capped[k], 1ull);
        }
    }
}

__global__ void __launch_bounds__(1024, 1) certify_cta256_kernel(const DevProblem P, const int32_t* __restrict__ cls,
                                                                 const int32_t count, const float2* __restrict__ msg) {
    using S = BigSmem;
    constexpr int D = kBigD;
    extern __shared__ __align__(16) unsigned char sm[];
    double2* tri_s = reinterpret_cast<double2*>(sm);
    RotC<double>* prm = reinterpret_cast<RotC<double>*>(sm + S::off_prm);
    int* idx0 = reinterpret_cast<int*>(sm + S::off_idx);
    int* idx1 = idx0 + D;
    unsigned short* tab = reinterpret_cast<unsigned short*>(sm + S::off_tab);
    double* red = reinterpret_cast<double*>(sm + S::off_red);
    const int t = threadIdx.x;
    double2* slot = reinterpret_cast<double2*>(P.big + (int64_t)blockIdx.x * P.big_slot);
    build_table<D, double>(tab);
    const int total = P.n_inst * count;
    for (int b = blockIdx.x; b < total; b += gridDim.x) {
        const int inst = b / count;
        const int r = cls[b % count];
        const RegionInfo R = P.reg[r];
        Split<double> A{tri_s, slot, S::ns64, D};
        __syncthreads();
        if (t < D) idx0[t] = t;
        assemble_packed<D, double>(P, R, inst, A, msg, nullptr, 0.0f, true);
        __syncthreads();
        double vr[D / 4], vi[D / 4];
        double norm2, off2;
        jacobi_cta<D, double, false>(A, prm, idx0, idx1, tab, red, vr, vi, P.st->cert_sweeps, 1e-28, norm2, off2);
        double lmin = A.dget(0).x;
        for (int i = 1; i < D; ++i) lmin = fmin(lmin, A.dget(i).x);
        lmin -= sqrt(off2);   // Weyl: a lower bound on lambda_min also when the sweep cap stopped it
        if (t == 0) {
            P.val64[(int64_t)inst * P.n_regions + r] = lmin;
            if (!isfinite(lmin)) atomicOr(P.err, DEV_ERR_NUMERIC);
            if (off2 > 1e-28 * norm2) atomicOr(P.err, DEV_ERR_NOCONV);
        }
    }
}

cudaError_t pass_cta256(const DevProblem& P, const PassIO& io, const int32_t* cls, int32_t count, int k, cudaStream_t s) {
    if (!P.big || P.big_slots <= 0) return cudaErrorInvalidValue;
    const int64_t blocks = std::min<int64_t>((int64_t)P.n_inst * count, P.big_slots);
    region_pass_cta256_kernel<<<(unsigned)blocks, 1024, BigSmem::bytes, s>>>(P, io, cls, count, k);
    return cudaGetLastError();
}

cudaError_t cert_cta256(const DevProblem& P, const int32_t* cls, int32_t count, const float2* msg, cudaStream_t s) {
    if (!P.big || P.big_slots <= 0) return cudaErrorInvalidValue;
    const int64_t blocks = std::min<int64_t>((int64_t)P.n_inst * count, P.big_slots);
    certify_cta256_kernel<<<(unsigned)blocks, 1024, BigSmem::bytes, s>>>(P, cls, count, msg);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Adjoint of the smoothed pass for D = 64 and 128 (see lrh_vjp.cu for the formulas): the
// eigenbasis is recomputed by the CTA Jacobi at the same point eta, then
//   Y = rho_bar V,  M = V^dagger Y,  X = M o K + (beta <rho_bar, rho> + q_bar) diag(p),
//   Z = V X,  theta_bar = Z V^dagger,
// four complex D x D products in TR x TC register tiles.  One D x D operand lives in shared
// memory (rho_bar, then M / X, then theta_bar) and V, Y / Z in the CTA's global scratch slot
// (2 D^2 complex, L2-resident while the CTA runs).  CTAs loop over the regions of the launch.
template <int D, typename FA, typename FB, typename FS>
__device__ __forceinline__ void cmm_tile(FA A, FB B, FS store) {
    constexpr int NT = CtaCfg<D>::NT, TR = CtaCfg<D>::TR, TC = CtaCfg<D>::TC, CS = D / TC;
    const int t = threadIdx.x;
    const int i0 = (t / CS) * TR, cb = t % CS;
    static_assert((D / TR) * CS == NT, "tile cover");
    float accr[TR][TC], acci[TR][TC];
#pragma unroll
    for (int a = 0; a < TR; ++a)
#pragma unroll
        for (int b = 0; b < TC; ++b) { accr[a][b] = 0.f; acci[a][b] = 0.f; }
    for (int k = 0; k < D; ++k) {
        float2 av[TR], bv[TC];
#pragma unroll
        for (int a = 0; a < TR; ++a) av[a] = A(i0 + a, k);
#pragma unroll
        for (int b = 0; b < TC; ++b) bv[b] = B(k, cb + CS * b);
#pragma unroll
        for (int a = 0; a < TR; ++a)
#pragma unroll
            for (int b = 0; b < TC; ++b) {
                accr[a][b] += av[a].x * bv[b].x - av[a].y * bv[b].y;
                acci[a][b] += av[a].x * bv[b].y + av[a].y * bv[b].x;
            }
    }
#pragma unroll
    for (int a = 0; a < TR; ++a)
#pragma unroll
        for (int b = 0; b < TC; ++b) store(i0 + a, cb + CS * b, make_float2(accr[a][b], acci[a][b]));
}

template <int D>
__global__ void __launch_bounds__(CtaCfg<D>::NT) vjp_cta_kernel(const DevProblem P, const int32_t* __restrict__ cls,
                                                                const int32_t count, float2* __restrict__ scratch) {
    using S = CtaSmem<D, float>;
    constexpr int NT = CtaCfg<D>::NT;
    constexpr int W = D / 4;
    constexpr int LD = D + 1;
    extern __shared__ __align__(16) unsigned char sm[];
    float2* buf = reinterpret_cast<float2*>(sm);
    RotC<float>* prm = reinterpret_cast<RotC<float>*>(sm + S::off_prm);
    int* idx0 = reinterpret_cast<int*>(sm + S::off_idx);
    int* idx1 = idx0 + D;
    unsigned short* tab = reinterpret_cast<unsigned short*>(sm + S::off_tab);
    float* lam = reinterpret_cast<float*>(sm + S::off_lam);
    float* pp = lam + D;
    float* red = reinterpret_cast<float*>(sm + S::off_red);
    const int t = threadIdx.x;
    float2* Vg = scratch + (int64_t)blockIdx.x * 2 * D * D;
    float2* Yg = Vg + D * D;
    const float th = (float)P.st->th3[P.st->t0 % 3];
    const float beta = (float)P.st->beta;
    build_table<D, float>(tab);
    const int total = P.n_inst * count;
    for (int b = blockIdx.x; b < total; b += gridDim.x) {
        const int inst = b / count;
        const int r = cls[b % count];
        const RegionInfo R = P.reg[r];
        Full<float> A{buf, D};
        __syncthreads();
        if (t < D) idx0[t] = A.sig(t);
        assemble_packed<D, float>(P, R, inst, A, P.nu, P.zeta, th, false);
        __syncthreads();
        const int row = vrow_of(t), chunk = vchunk_of(t);
        float vr[W], vi[W];
#pragma unroll
        for (int m = 0; m < W; ++m) { vr[m] = (chunk * W + m == row) ? 1.f : 0.f; vi[m] = 0.f; }
        float norm2, off2;
        jacobi_cta<D, float, true>(A, prm, idx0, idx1, tab, red, vr, vi, P.st->max_sweeps, 1e-12f, norm2, off2);
        if (t < D) lam[t] = A.dget(A.sig(t)).x;
        __syncthreads();
        float lmin = lam[0];
        for (int i = 1; i < D; ++i) lmin = fminf(lmin, lam[i]);
        float Z = 0.f;
        for (int i = 0; i < D; ++i) Z += expf(-beta * (lam[i] - lmin));
        if (t < D) pp[t] = expf(-beta * (lam[t] - lmin)) / Z;
#pragma unroll
        for (int m = 0; m < W; ++m) Vg[row * D + chunk * W + m] = make_float2(vr[m], vi[m]);
        __syncthreads();
        // rho_bar (general D x D): the gather of theta with h = 0 applied to g_bar
        const int64_t mbase = (int64_t)inst * P.msg_elems;
        for (int e = t; e < D * D; e += NT) {
            const int i = e / D, j = e % D;
            float re = 0.f, im = 0.f;
            for (int q = R.child_begin; q < R.child_end; ++q) {
                const PairInfo pi = P.child_info[q];
                if (((i ^ j) & ~pi.mask) != 0) continue;
                const int Df = 1 << pi.kf;
                const float2 m = P.gbar[mbase + pi.off + (int64_t)pext8(i, pi.mask) * Df + pext8(j, pi.mask)];
                re -= m.x; im -= m.y;
            }
            for (int q = R.parent_begin; q < R.parent_end; ++q) {
                const float2 m = P.gbar[mbase + P.parent_info[q].off + e];
                re += m.x; im += m.y;
            }
            buf[i * LD + j] = make_float2(re, im);
        }
        __syncthreads();
        // (1) Y = rho_bar V
        cmm_tile<D>([&](int i, int k) { return buf[i * LD + k]; }, [&](int k, int j) { return Vg[k * D + j]; },
                    [&](int i, int j, float2 v) { Yg[i * D + j] = v; });
        __syncthreads();
        // (2) M = V^dagger Y (into shared memory; rho_bar is no longer needed)
        cmm_tile<D>([&](int i, int k) { const float2 v = Vg[k * D + i]; return make_float2(v.x, -v.y); },
                    [&](int k, int j) { return Yg[k * D + j]; }, [&](int i, int j, float2 v) { buf[i * LD + j] = v; });
        __syncthreads();
        // <rho_bar, rho> = sum_k p_k Re M_kk;  X = M o K + (beta <rho_bar, rho> + q_bar) diag(p)
        float part = 0.f;
        for (int k = t; k < D; k += NT) part += pp[k] * buf[k * LD + k].x;
        const float inner = block_sum<NT>(part, red);
        const float coef = beta * inner + (float)P.qbar[inst];
        for (int e = t; e < D * D; e += NT) {
            const int i = e / D, j = e % D;
            const float kv = kdd(lam[i], lam[j], pp[i], pp[j], beta);
            float2 x = buf[i * LD + j];
            x.x *= kv; x.y *= kv;
            if (i == j) x.x += coef * pp[i];
            buf[i * LD + j] = x;
        }
        __syncthreads();
        // (3) Z = V X (into the slot; Y is no longer needed)
        cmm_tile<D>([&](int i, int k) { return Vg[i * D + k]; }, [&](int k, int j) { return buf[k * LD + j]; },
                    [&](int i, int j, float2 v) { Yg[i * D + j] = v; });
        __syncthreads();
        // (4) theta_bar = Z V^dagger
        cmm_tile<D>([&](int i, int k) { return Yg[i * D + k]; },
                    [&](int k, int j) { const float2 v = Vg[j * D + k]; return make_float2(v.x, -v.y); },
                    [&](int i, int j, float2 v) { buf[i * LD + j] = v; });
        __syncthreads();
        // exactly Hermitian (upper triangle as computed), out to theta_bar and onto the children
        float2* dst = P.thb + (int64_t)inst * P.all_elems + R.all_off;
        for (int e = t; e < D * D; e += NT) {
            const int i = e / D, j = e % D;
            float2 v = i <= j ? buf[i * LD + j] : buf[j * LD + i];
            if (i > j) v.y = -v.y;
            if (i == j) v.y = 0.f;
            dst[e] = v;
        }
        __syncthreads();
        float2* trb = P.tr + (int64_t)inst * P.msg_elems;
        for (int q = R.child_begin; q < R.child_end; ++q) {
            const PairInfo pi = P.child_info[q];
            const int M = pi.mask, Mc = (D - 1) & ~M, kf = pi.kf, Df = 1 << kf, nrest = D >> kf;
            for (int o = t; o < Df * Df; o += NT) {
                const int ra = pdep8(o >> kf, M), rbb = pdep8(o & (Df - 1), M);
                float sr = 0.f, si = 0.f;
                for (int c = 0; c < nrest; ++c) {
                    const int x = pdep8(c, Mc);
                    const float2 v = dst[(ra | x) * D + (rbb | x)];
                    sr += v.x; si += v.y;
                }
                trb[pi.off + o] = make_float2(sr, si);
            }
        }
    }
}

template <int D>
cudaError_t pass_cta(const DevProblem& P, const PassIO& io, const int32_t* cls, int32_t count, int k, cudaStream_t s) {
    const int64_t blocks = (int64_t)P.n_inst * count;
    region_pass_cta_kernel<D><<<(unsigned)blocks, CtaCfg<D>::NT, CtaSmem<D, float>::bytes, s>>>(P, io, cls, count, k);
    return cudaGetLastError();
}

template <int D>
cudaError_t cert_cta(const DevProblem& P, const int32_t* cls, int32_t count, const float2* msg, cudaStream_t s) {
    const int64_t blocks = (int64_t)P.n_inst * count;
    certify_cta_kernel<D><<<(unsigned)blocks, CtaCfg<D>::NT, CtaSmem<D, double>::bytes, s>>>(P, cls, count, msg);
    return cudaGetLastError();
}

}  // namespace

cudaError_t prepare_cta_kernels() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(region_pass_cta_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)CtaSmem<64, float>::bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(region_pass_cta_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)CtaSmem<128, float>::bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(vjp_cta_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)CtaSmem<64, float>::bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(vjp_cta_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)CtaSmem<128, float>::bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(region_pass_cta256_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)BigSmem::bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(certify_cta256_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)BigSmem::bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(certify_cta_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)CtaSmem<64, double>::bytes)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(certify_cta_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)CtaSmem<128, double>::bytes);
}

cudaError_t launch_region_pass_cta(const DevProblem& P, const PassIO& io, int k, const int32_t* cls, int32_t count,
                                   cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    if (k == 6) return pass_cta<64>(P, io, cls, count, k, s);
    if (k == 7) return pass_cta<128>(P, io, cls, count, k, s);
    if (k == 8) return pass_cta256(P, io, cls, count, k, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_certify_cta(const DevProblem& P, int k, const int32_t* cls, int32_t count, const float2* msg,
                               cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    if (k == 6) return cert_cta<64>(P, cls, count, msg, s);
    if (k == 7) return cert_cta<128>(P, cls, count, msg, s);
    if (k == 8) return cert_cta256(P, cls, count, msg, s);
    return cudaErrorInvalidValue;
}

cudaError_t vjp_cta_slots(int k, int* slots) {
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if (k == 6) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, vjp_cta_kernel<64>, CtaCfg<64>::NT, CtaSmem<64, float>::bytes);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, vjp_cta_kernel<128>, CtaCfg<128>::NT, CtaSmem<128, float>::bytes);
    if (e != cudaSuccess) return e;
    *slots = sms * std::max(1, occ);
    return cudaSuccess;
}

cudaError_t launch_vjp_cta(const DevProblem& P, int k, const int32_t* cls, int32_t count, float2* scratch, int slots,
                           cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((int64_t)P.n_inst * count, slots);
    if (k == 6) vjp_cta_kernel<64><<<(unsigned)blocks, CtaCfg<64>::NT, CtaSmem<64, float>::bytes, s>>>(P, cls, count, scratch);
    else if (k == 7) vjp_cta_kernel<128><<<(unsigned)blocks, CtaCfg<128>::NT, CtaSmem<128, float>::bytes, s>>>(P, cls, count, scratch);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

int64_t big_slot_elems(int log_sweeps) {
    return kBigOffLog + 2 * (int64_t)log_sweeps * (kBigD - 1) * kBigN;   // a RotC<float> is two complex64
}

cudaError_t big_launch_slots(int* slots) {
    int dev = 0, sms = 0, occ_p = 0, occ_c = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_p, region_pass_cta256_kernel, 1024, BigSmem::bytes)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_c, certify_cta256_kernel, 1024, BigSmem::bytes)) != cudaSuccess) return e;
    *slots = sms * std::max(1, std::max(occ_p, occ_c));
    return cudaSuccess;
}

}  // namespace lrh
