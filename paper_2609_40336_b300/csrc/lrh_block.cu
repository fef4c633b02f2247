// Per-class launches of the 2x2-block region pass (D = 8, 16); the device code is in lrh_block.cuh.
#include "lrh_block.cuh"

namespace lrh {

namespace {

using blk::BlkSmem;
using blk::region_pass_blk_impl;
using dev::advance_theta;

template <int D> struct BlkCap { static constexpr int v = D == 16 ? 128 : 96; };

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) region_pass_w16_kernel(const DevProblem P, const PassIO io,
                                                                const int32_t* __restrict__ cls, const int32_t count,
                                                                const int k) {
    if (io.writer && blockIdx.x == 0 && threadIdx.x == 0) advance_theta(P, io);
    blk::region_pass_w16_impl<BLOCK>(P, io, cls, count, k, blockIdx.x);
}

template <int BLOCK>
cudaError_t w16_attr() {
    return cudaFuncSetAttribute(region_pass_w16_kernel<BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)blk::W16Smem<BLOCK>::bytes);
}

template <int BLOCK>
cudaError_t w16_launch(const DevProblem& P, const PassIO& io, const int32_t* cls, int32_t count, int k, cudaStream_t s) {
    constexpr int G = BLOCK / 32;
    const int64_t units = (int64_t)P.n_inst * count;
    const int64_t blocks = (units + G - 1) / G;
    region_pass_w16_kernel<BLOCK><<<(unsigned)blocks, BLOCK, blk::W16Smem<BLOCK>::bytes, s>>>(P, io, cls, count, k);
    return cudaGetLastError();
}

template <int D, int BLOCK>
__global__ void __launch_bounds__(BLOCK) __maxnreg__(BlkCap<D>::v)
    region_pass_blk_kernel(const DevProblem P, const PassIO io, const int32_t* __restrict__ cls, const int32_t count,
                           const int k) {
    if (io.writer && blockIdx.x == 0 && threadIdx.x == 0) advance_theta(P, io);
    region_pass_blk_impl<D, BLOCK>(P, io, cls, count, k, blockIdx.x);
}

template <int D, int BLOCK>
cudaError_t blk_attr() {
    return cudaFuncSetAttribute(region_pass_blk_kernel<D, BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)BlkSmem<D, BLOCK>::bytes);
}

template <int D, int BLOCK>
cudaError_t blk_launch(const DevProblem& P, const PassIO& io, const int32_t* cls, int32_t count, int k, cudaStream_t s) {
    constexpr int G = BLOCK / D;
    const int64_t units = (int64_t)P.n_inst * count;
    const int64_t blocks = (units + G - 1) / G;
    region_pass_blk_kernel<D, BLOCK><<<(unsigned)blocks, BLOCK, BlkSmem<D, BLOCK>::bytes, s>>>(P, io, cls, count, k);
    return cudaGetLastError();
}

template <int D>
cudaError_t blk_launch_D(const DevProblem& P, const PassIO& io, const int32_t* cls, int32_t count, int k, cudaStream_t s,
                         int threads) {
    if (threads == 64) return blk_launch<D, 64>(P, io, cls, count, k, s);
    if (threads == 256) return blk_launch<D, 256>(P, io, cls, count, k, s);
    return blk_launch<D, 128>(P, io, cls, count, k, s);
}

}  // namespace

cudaError_t prepare_blk_kernels() {
    cudaError_t e;
    if ((e = blk_attr<8, 64>()) != cudaSuccess || (e = blk_attr<8, 128>()) != cudaSuccess ||
        (e = blk_attr<8, 256>()) != cudaSuccess || (e = blk_attr<16, 64>()) != cudaSuccess ||
        (e = blk_attr<16, 128>()) != cudaSuccess || (e = blk_attr<16, 256>()) != cudaSuccess ||
        (e = w16_attr<64>()) != cudaSuccess || (e = w16_attr<128>()) != cudaSuccess || (e = w16_attr<256>()) != cudaSuccess)
        return e;
    return cudaSuccess;
}

cudaError_t launch_region_pass_w16(const DevProblem& P, const PassIO& io, const int32_t* cls, int32_t count,
                                   cudaStream_t s, int threads) {
    if (count <= 0) return cudaSuccess;
    if (threads == 64) return w16_launch<64>(P, io, cls, count, 4, s);
    if (threads == 256) return w16_launch<256>(P, io, cls, count, 4, s);
    return w16_launch<128>(P, io, cls, count, 4, s);
}

cudaError_t launch_region_pass_blk(const DevProblem& P, const PassIO& io, int k, const int32_t* cls, int32_t count,
                                   cudaStream_t s, int threads) {
    if (count <= 0) return cudaSuccess;
    if (k == 3) return blk_launch_D<8>(P, io, cls, count, k, s, threads);
    if (k == 4) return blk_launch_D<16>(P, io, cls, count, k, s, threads);
    return cudaErrorInvalidValue;
}

}  // namespace lrh
