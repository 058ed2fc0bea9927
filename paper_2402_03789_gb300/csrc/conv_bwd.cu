// Per-edge adjoint of the convolution (the instantiation behind the
// convolution entry points and the halo emulation), and the conversion of the
// fixed-point dE/dx sums.
#include "conv_bwd.cuh"

namespace sn {

// dE/dx from its fixed-point sums; a sum that received the sentinel becomes
// NaN and sets flags[FLAG_GX_OVERFLOW] (flags may be null).
__global__ void gx_from_fixed_kernel(int64_t n, const unsigned long long* __restrict__ q, float* __restrict__ gx,
                                     int* flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long v = (long long)q[i];
    const long long lim = 1LL << 56;
    if (v >= lim || v <= -lim) {
        gx[i] = __int_as_float(0x7fc00000);
        if (flags) atomicOr(flags + FLAG_GX_OVERFLOW, 1);
    } else {
        gx[i] = (float)((double)v * (1.0 / 68719476736.0));
    }
}

void launch_gx_from_fixed(size_t nx, const unsigned long long* gxq, float* gx, int* flags, cudaStream_t st) {
    if (nx) gx_from_fixed_kernel<<<(unsigned)((nx + 255) / 256), 256, 0, st>>>((int64_t)nx, gxq, gx, flags);
}

sevennet_status conv_configure_bwd(int H, size_t need) { return conv_configure_bwd_mode<false>(H, need); }

void launch_conv_bwd(const LayerDev& L, int H, sevennet_precision prec, int64_t n_atoms,
                     int64_t n_edges, const int* row_ptr, const int* dst, const int* src,
                     const float4* geom, const float* x, const float* gm, float* gx,
                     unsigned long long* gxq, int* flags, float* gd, cudaStream_t st) {
    const size_t nx = (size_t)std::max<int64_t>(n_atoms, 0) * L.conv.x_dim;
    if (!gx) gxq = nullptr;                      // the kernel then skips the dE/dx sums
    if (gxq && nx) cudaMemsetAsync(gxq, 0, nx * sizeof(unsigned long long), st);
    conv_bwd_dispatch<false>(L, H, prec == SEVENNET_BF16, n_edges, row_ptr + std::max<int64_t>(n_atoms, 0), dst,
                             src, geom, nullptr, x, gm, gxq, gd, st);
    if (gxq) launch_gx_from_fixed(nx, gxq, gx, flags, st);
}

}  // namespace sn
