// Forward tensor-product convolution of one interaction block (Eq. 3,
// Figure 2b): radial MLP, CG tensor product and the segmented sum into
// receivers, fused per 16-edge chunk.  Shared phases live in conv_common.cuh.
#include "conv_common.cuh"

namespace sn {

// One group = one path and CPL channels per lane (32*CPL channels per warp).
// The lane walks the chunk's edges, keeps the running message of the current
// receiver in registers and writes it once when the receiver changes.  The
// edge's G matrix and the address arithmetic serve all CPL channels.
template <int L1, int L2, int L3, int CPL>
__device__ __forceinline__ void tp_fwd_group(const PathDesc& P, int u0, int ne,
                                             const float* s_w, int Wpad, const float* s_G, int nG,
                                             const int* s_src, const int* s_dst, const int* s_first,
                                             const float* __restrict__ x, int x_dim,
                                             float* __restrict__ m, int m_dim) {
    constexpr int N1 = 2 * L1 + 1, N3 = 2 * L3 + 1;
    constexpr int PF = (CPL * N1 <= 1) ? 16 : (CPL * N1 <= 2) ? 8 : (CPL * N1 <= 4) ? 4 : 2;   // gathers in flight
    const int col = P.col0 + u0;
    const int mul = P.mul;
    const float* xb = x + P.x_off + u0;
    float* mb = m + P.m_off + P.m_ch0 + u0;
    // A receiver that started in this CTA's previous chunk was written there by
    // this same thread; its partial sum seeds the accumulator, and the load
    // overlaps the first gathers.
    float acc[CPL][N3];
    if (!s_first[0]) {
        const float* mp = mb + (size_t)s_dst[0] * m_dim;
#pragma unroll
        for (int k = 0; k < CPL; ++k)
#pragma unroll
            for (int c = 0; c < N3; ++c) acc[k][c] = mp[c * P.m_mul + 32 * k];
    } else {
#pragma unroll
        for (int k = 0; k < CPL; ++k)
#pragma unroll
            for (int c = 0; c < N3; ++c) acc[k][c] = 0.0f;
    }
    int cur = s_dst[0];
    auto flush = [&](int v) {
        float* mp = mb + (size_t)v * m_dim;
#pragma unroll
        for (int k = 0; k < CPL; ++k)
#pragma unroll
            for (int c = 0; c < N3; ++c) mp[c * P.m_mul + 32 * k] = acc[k][c];
    };
    for (int e0 = 0; e0 < ne; e0 += PF) {
        float xv[PF][CPL][N1];
#pragma unroll
        for (int q = 0; q < PF; ++q) {
            const int e = min(e0 + q, ne - 1);
            const float* xr = xb + (size_t)s_src[e] * x_dim;
#pragma unroll
            for (int k = 0; k < CPL; ++k)
#pragma unroll
                for (int a = 0; a < N1; ++a) xv[q][k][a] = __ldg(xr + a * mul + 32 * k);
        }
#pragma unroll
        for (int q = 0; q < PF; ++q) {
            const int e = e0 + q;
            if (e >= ne) break;
            const int v = s_dst[e];
            if (v != cur) {
                flush(cur);
                cur = v;
#pragma unroll
                for (int k = 0; k < CPL; ++k)
#pragma unroll
                    for (int c = 0; c < N3; ++c) acc[k][c] = 0.0f;
            }
            float G[((N1 * N3 + 3) / 4) * 4];
            load_G<N1 * N3>(s_G + e * nG + P.g_off, G);
            const float* wr = s_w + e * Wpad + col;
#pragma unroll
            for (int k = 0; k < CPL; ++k) {
                const float wv = wr[32 * k];
#pragma unroll
                for (int c = 0; c < N3; ++c) {
                    float tt = 0.0f;
#pragma unroll
                    for (int a = 0; a < N1; ++a) tt = fmaf(xv[q][k][a], G[a * N3 + c], tt);
                    acc[k][c] = fmaf(wv, tt, acc[k][c]);
                }
            }
        }
    }
    if (ne > 0) flush(cur);
}

template <int H, bool BF>
__global__ void __launch_bounds__(CONV_THREADS, 2)
conv_fwd_kernel(const ConvDesc D, const float* __restrict__ W1, const float* __restrict__ W2,
                const float* __restrict__ W3, const __nv_bfloat16* __restrict__ W3T_h,
                const __nv_bfloat16* __restrict__ W2T_h, int n_atoms, int n_edges,
                const int* __restrict__ row_ptr, const int* __restrict__ dst,
                const int* __restrict__ src, const float4* __restrict__ geom,
                const float* __restrict__ x, float* __restrict__ m) {
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    const ConvSmem L = conv_smem_layout(D.Wpad, H, D.nG, false);
    __shared__ int s_range[2];
    cta_range(n_atoms, n_edges, row_ptr, s_range);
    const int v0 = s_range[0], v1 = s_range[1];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    // receivers without edges get zero messages
    for (int v = v0 + warp; v < v1; v += CONV_WARPS) {
        if (row_ptr[v] == row_ptr[v + 1]) {
            for (int i = lane; i < D.m_dim; i += 32) m[(size_t)v * D.m_dim + i] = 0.0f;
        }
    }
    const int E0 = row_ptr[v0], E1 = row_ptr[v1];
    const int* s_src = reinterpret_cast<const int*>(smem + L.src);
    const int* s_dst = reinterpret_cast<const int*>(smem + L.dst);
    const int* s_first = reinterpret_cast<const int*>(smem + L.first);
    EdgePrefetch pf;
    pf.fetch(E0, E1, dst, src, geom, row_ptr);
    for (int c0 = E0; c0 < E1; c0 += EC) {
        const int ne = min(EC, E1 - c0);
        __syncthreads();
        chunk_prologue<H, BF>(D, L, smem, c0, ne, pf, W1, W2, W2T_h);
        pf.fetch(c0 + EC, E1, dst, src, geom, row_ptr);   // next chunk's edges, in flight meanwhile
        if constexpr (BF) chunk_w_gemm_bf16<H>(D, L, smem, W3T_h);
        else chunk_w_gemm_f32<H>(D, L, smem, W3);
        for (int s = 0; s < D.n_slots[warp]; ++s) {
            const int g = D.slot_group[warp][s];
            const PathDesc& P = D.paths[g >> 8];
            const int lc = g & 3;                      // log2 of channels per lane
            const int u0 = ((g >> 2) & 63) * (32 << lc) + lane;
            switch (P.kind * 3 + lc) {
#define SN_F1(a, b, c, l)                                                                          \
                case coupling_kind(a, b, c) * 3 + l:                                               \
                    if constexpr (fwd_cpl_compiled(H, a, 1 << l))                                  \
                        tp_fwd_group<a, b, c, (1 << l)>(P, u0, ne, smem + L.w, D.Wpad, smem + L.G, \
                                                        D.nG, s_src, s_dst, s_first, x, D.x_dim, m, \
                                                        D.m_dim);                                  \
                    break;
#define SN_F(a, b, c) SN_F1(a, b, c, 0) SN_F1(a, b, c, 1) SN_F1(a, b, c, 2)
                SN_F(0, 0, 0) SN_F(0, 1, 1) SN_F(0, 2, 2)
                SN_F(1, 0, 1) SN_F(1, 1, 0) SN_F(1, 1, 1) SN_F(1, 1, 2) SN_F(1, 2, 1) SN_F(1, 2, 2)
                SN_F(2, 0, 2) SN_F(2, 1, 1) SN_F(2, 1, 2) SN_F(2, 2, 0) SN_F(2, 2, 1) SN_F(2, 2, 2)
#undef SN_F
#undef SN_F1
                default: break;
            }
        }
    }
}

// ------------------------------------------------------------- edge preparation
__global__ void prep_dst_kernel(int64_t n, const int* __restrict__ row_ptr, int* __restrict__ dst) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    for (int e = row_ptr[v]; e < row_ptr[v + 1]; ++e) dst[e] = (int)v;
}

__global__ void prep_geom_kernel(int64_t E, const float* __restrict__ d, float4* __restrict__ geom) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const float x = d[e * 3], y = d[e * 3 + 1], z = d[e * 3 + 2];
    geom[e] = make_float4(x, y, z, sqrtf(x * x + y * y + z * z));
}

void conv_prepare_edges(int64_t n_atoms, int64_t n_edges, const int* row_ptr, const float* d, int* dst,
                        float4* geom, cudaStream_t st) {
    if (n_atoms > 0) prep_dst_kernel<<<(unsigned)((n_atoms + 255) / 256), 256, 0, st>>>(n_atoms, row_ptr, dst);
    if (n_edges > 0) prep_geom_kernel<<<(unsigned)((n_edges + 255) / 256), 256, 0, st>>>(n_edges, d, geom);
}

// ------------------------------------------------------------- launcher
size_t conv_smem_bytes(const ConvDesc& D, int H, bool bwd) { return smem_bytes(D, H, bwd); }

sevennet_status conv_configure_fwd(int H, size_t need) {
    static size_t granted[2][2] = {{0, 0}, {0, 0}};
    const int hi = H == 64 ? 1 : 0;
    if (H == 64) {
        SN_TRY(conv_set_smem((const void*)conv_fwd_kernel<64, false>, need, &granted[hi][0]));
        SN_TRY(conv_set_smem((const void*)conv_fwd_kernel<64, true>, need, &granted[hi][1]));
    } else if (H == 32) {
        SN_TRY(conv_set_smem((const void*)conv_fwd_kernel<32, false>, need, &granted[hi][0]));
        SN_TRY(conv_set_smem((const void*)conv_fwd_kernel<32, true>, need, &granted[hi][1]));
    } else {
        set_error("radial MLP hidden width must be 32 or 64");
        return SEVENNET_EINVAL;
    }
    return SEVENNET_OK;
}

void launch_conv_fwd(const LayerDev& L, int H, sevennet_precision prec, int64_t n_atoms,
                     int64_t n_edges, const int* row_ptr, const int* dst, const int* src,
                     const float4* geom, const float* x, float* m, cudaStream_t st) {
    const int grid = conv_grid(n_atoms);
    const size_t sm = smem_bytes(L.conv, H, false);
    const bool bf = prec == SEVENNET_BF16;
#define SN_LF(HH, BB) conv_fwd_kernel<HH, BB><<<grid, CONV_THREADS, sm, st>>>(                     \
        L.conv, L.mlp0, L.mlp1, L.mlp2, L.mlp2h, L.mlp1Th, (int)n_atoms, (int)n_edges, row_ptr, dst, src, geom, x, m)
    if (H == 64) { if (bf) SN_LF(64, true); else SN_LF(64, false); }
    else         { if (bf) SN_LF(32, true); else SN_LF(32, false); }
#undef SN_LF
}

}  // namespace sn
