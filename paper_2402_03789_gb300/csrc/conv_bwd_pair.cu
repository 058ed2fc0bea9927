// Adjoint of the convolution over unordered pairs of edges (the model's
// evaluation path): the radial MLP, the G matrices and their adjoints once per
// pair, the tensor product once per direction (conv_bwd.cuh).
#include "conv_bwd.cuh"

namespace sn {

sevennet_status conv_configure_bwd_pair(int H, size_t need) { return conv_configure_bwd_mode<true>(H, need); }

void launch_conv_bwd_pair(const LayerDev& L, int H, sevennet_precision prec, int64_t n_atoms, int64_t n_pairs,
                          const int* pair_ptr, const int* p_dst, const int* p_src, const float4* p_geom,
                          const int* p_e, const float* x, const float* gm, float* gx, unsigned long long* gxq,
                          int* flags, float* gd, cudaStream_t st) {
    const size_t nx = (size_t)std::max<int64_t>(n_atoms, 0) * L.conv.x_dim;
    if (!gx) gxq = nullptr;
    if (gxq && nx) cudaMemsetAsync(gxq, 0, nx * sizeof(unsigned long long), st);
    conv_bwd_dispatch<true>(L, H, prec == SEVENNET_BF16, n_pairs, pair_ptr + std::max<int64_t>(n_atoms, 0), p_dst,
                            p_src, p_geom, p_e, x, gm, gxq, gd, st);
    if (gxq) launch_gx_from_fixed(nx, gxq, gx, flags, st);
}

}  // namespace sn
