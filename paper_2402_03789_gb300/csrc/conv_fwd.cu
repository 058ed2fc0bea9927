// Forward tensor-product convolution of one interaction block (Eq. 3,
// Figure 2b): radial MLP, CG tensor product and the segmented sum into
// receivers, fused per 16-edge chunk.  Shared phases live in conv_common.cuh.
#include "conv_common.cuh"

namespace sn {

// Forward gathers: a rolling one-edge-ahead prefetch (one copy of the edge
// body) or PF edges unrolled together.
constexpr bool FWD_ROLL = false;

template <int L1, int LMAX, int KIND>
struct FwdSets {
    static constexpr PathSets sets = fwd_path_sets(L1, LMAX, KIND);
};

// Offset of path i of the l1 list inside the running sums of its set.
template <int L1, int LMAX, int KIND>
__host__ __device__ constexpr int fwd_acc_off(int j, int i) {
    const PathList p = path_list(L1, LMAX, KIND);
    int o = 0;
    for (int k = fwd_path_sets(L1, LMAX, KIND).b[j]; k < i; ++k) o += 2 * p.l3[k] + 1;
    return o;
}

// One work set: the paths [I0, I1) of input irrep L1 for CPL channels per lane
// (channels u0 + 32 k).  The lane walks the chunk's edges, gathers x_src[L1]
// once per edge for all paths of the set, keeps the running messages of the
// current receiver in registers and writes them once when the receiver
// changes.  A receiver that started in this CTA's previous chunk was written
// there by this same thread; its partial sums seed the registers, loaded
// before the first gathers so the two overlap.
template <int L1, int LMAX, int KIND, int J, int CPL, typename WT>
__device__ __forceinline__ void tp_fwd_set(const ConvDesc& D, int u0, int ne, const WT* s_w,
                                           const float* s_G, const int* s_src, const int* s_dst,
                                           const int* s_first, const float* __restrict__ x,
                                           float* __restrict__ m) {
    using BP = BlockPaths<L1, LMAX, KIND>;
    constexpr int I0 = FwdSets<L1, LMAX, KIND>::sets.b[J];
    constexpr int I1 = FwdSets<L1, LMAX, KIND>::sets.b[J + 1];
    constexpr int NP = I1 - I0;
    constexpr int N1 = 2 * L1 + 1;
    constexpr int NACC = fwd_set_nacc(L1, LMAX, KIND, J);
    constexpr int PF = (CPL * N1 <= 2) ? 4 : 2;           // edges whose gathers are in flight together
    const int mul = D.mul_in[L1];
    const int Wpad = sizeof(WT) == 2 ? D.WpadB : D.Wpad, nG = D.nG, m_dim = D.m_dim, x_dim = D.x_dim;
    const float* xb = x + D.x_off[L1] + u0;
    float acc[CPL][NACC];
    auto rows = [&](int v, auto&& f) {        // f(path P, acc offset, N3) for every path of the set
        static_for<NP>([&](auto I) {
            constexpr int i = I0 + decltype(I)::value;
            constexpr int N3 = 2 * BP::list.l3[i] + 1;
            constexpr int off = fwd_acc_off<L1, LMAX, KIND>(J, i);
            const PathDesc& P = D.paths[BP::begin + i];
            f(m + (size_t)v * m_dim + P.m_off + P.m_ch0 + u0, P.m_mul, off, std::integral_constant<int, N3>{});
        });
    };
    if (!s_first[0]) {
        rows(s_dst[0], [&](const float* mp, int mm, int off, auto n3) {
#pragma unroll
            for (int k = 0; k < CPL; ++k)
#pragma unroll
                for (int c = 0; c < decltype(n3)::value; ++c) acc[k][off + c] = mp[c * mm + 32 * k];
        });
    } else {
#pragma unroll
        for (int k = 0; k < CPL; ++k)
#pragma unroll
            for (int c = 0; c < NACC; ++c) acc[k][c] = 0.0f;
    }
    int cur = s_dst[0];
    auto flush = [&](int v) {
        rows(v, [&](const float* mp, int mm, int off, auto n3) {
            float* mw = const_cast<float*>(mp);
#pragma unroll
            for (int k = 0; k < CPL; ++k)
#pragma unroll
                for (int c = 0; c < decltype(n3)::value; ++c) mw[c * mm + 32 * k] = acc[k][off + c];
        });
    };
    // per edge: the running sums of every path of the set, for CPL channels
    auto edge = [&](int e, const float (&xv)[CPL][N1]) {
        const int v = s_dst[e];
        if (v != cur) {
            flush(cur);
            cur = v;
#pragma unroll
            for (int k = 0; k < CPL; ++k)
#pragma unroll
                for (int c = 0; c < NACC; ++c) acc[k][c] = 0.0f;
        }
        static_for<NP>([&](auto I) {
            constexpr int i = I0 + decltype(I)::value;
            constexpr int N3 = 2 * BP::list.l3[i] + 1;
            constexpr int off = fwd_acc_off<L1, LMAX, KIND>(J, i);
            const PathDesc& P = D.paths[BP::begin + i];
            float G[((N1 * N3 + 3) / 4) * 4];
            load_G<N1 * N3>(s_G + e * nG + P.g_off, G);
            const WT* wr = s_w + e * Wpad + P.col0 + u0;
#pragma unroll
            for (int k = 0; k < CPL; ++k) {
                const float wv = wload(wr + 32 * k);
#pragma unroll
                for (int c = 0; c < N3; ++c) {
                    float tt = 0.0f;
#pragma unroll
                    for (int a = 0; a < N1; ++a) tt = fmaf(xv[k][a], G[a * N3 + c], tt);
                    acc[k][off + c] = fmaf(wv, tt, acc[k][off + c]);
                }
            }
        });
    };
    auto gather = [&](int e, float (&xv)[CPL][N1]) {
        const float* xr = xb + (size_t)s_src[e] * x_dim;
#pragma unroll
        for (int k = 0; k < CPL; ++k)
#pragma unroll
            for (int a = 0; a < N1; ++a) xv[k][a] = __ldg(xr + a * mul + 32 * k);
    };
    if constexpr (FWD_ROLL) {
        // one copy of the edge body; the next edge's gathers are in flight meanwhile
        float xn[CPL][N1];
        if (ne > 0) gather(0, xn);
#pragma unroll 1
        for (int e = 0; e < ne; ++e) {
            float xv[CPL][N1];
#pragma unroll
            for (int k = 0; k < CPL; ++k)
#pragma unroll
                for (int a = 0; a < N1; ++a) xv[k][a] = xn[k][a];
            if (e + 1 < ne) gather(e + 1, xn);
            edge(e, xv);
        }
    } else {
        for (int e0 = 0; e0 < ne; e0 += PF) {
            float xv[PF][CPL][N1];
#pragma unroll
            for (int q = 0; q < PF; ++q) gather(min(e0 + q, ne - 1), xv[q]);
#pragma unroll
            for (int q = 0; q < PF; ++q) {
                if (e0 + q >= ne) break;
                edge(e0 + q, xv[q]);
            }
        }
    }
    if (ne > 0) flush(cur);
}

// Phase E of the forward: every warp runs its work sets over the chunk.
template <int H, int LMAX, int KIND, typename WT>
__device__ __forceinline__ void tp_fwd_chunk(const ConvDesc& D, int ne, const WT* s_w, const float* s_G,
                                             const int* s_src, const int* s_dst, const int* s_first,
                                             const float* __restrict__ x, float* __restrict__ m) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int s = 0; s < D.n_slots[warp]; ++s) {
        const int g = D.slot_group[warp][s];
        const int lc = g & 3, ub = (g >> 2) & 63, set = (g >> 8) & 7, l1 = (g >> 11) & 3;
        const int u0 = ub * (32 << lc) + lane;
        static_for<LMAX + 1>([&](auto L) {
            constexpr int L1 = decltype(L)::value;
            static_for<FWD_MAX_SETS>([&](auto Jc) {
                constexpr int J = decltype(Jc)::value;
                if constexpr (J < FwdSets<L1, LMAX, KIND>::sets.n) {
                    constexpr int NACC = fwd_set_nacc(L1, LMAX, KIND, J);
                    static_for<3>([&](auto Cc) {
                        constexpr int LC = decltype(Cc)::value;
                        if constexpr (fwd_cpl_compiled(H, L1, NACC, 1 << LC)) {
                            if (l1 == L1 && set == J && lc == LC)
                                tp_fwd_set<L1, LMAX, KIND, J, (1 << LC), WT>(D, u0, ne, s_w, s_G, s_src, s_dst,
                                                                        s_first, x, m);
                        }
                    });
                }
            });
        });
    }
}

template <int H, bool BF, int LMAX>
__global__ void __launch_bounds__(CONV_THREADS, conv_ctas_per_sm(LMAX))
conv_fwd_kernel(const ConvDesc D, const float* __restrict__ W1, const float* __restrict__ W2,
                const float* __restrict__ W3, const __nv_bfloat16* __restrict__ W3T_h,
                const __nv_bfloat16* __restrict__ W2T_h, int n_atoms, int n_edges,
                const int* __restrict__ row_ptr, const int* __restrict__ dst,
                const int* __restrict__ src, const float4* __restrict__ geom,
                const float* __restrict__ x, float* __restrict__ m) {
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    const ConvSmem L = conv_smem_layout(D.Wpad, D.WpadB, H, D.nG, D.ys, false, BF);
    using WT = typename WTile<BF>::T;
    const WT* s_w = reinterpret_cast<const WT*>(smem + L.w);
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
    load_W1<H>(D, L, smem, W1);
    EdgePrefetch pf;
    pf.fetch(E0, E1, dst, src, geom, row_ptr);
    for (int c0 = E0; c0 < E1; c0 += EC) {
        const int ne = min(EC, E1 - c0);
        __syncthreads();
        chunk_prologue<H, BF, LMAX>(D, L, smem, c0, ne, pf, W2, W2T_h);
        pf.fetch(c0 + EC, E1, dst, src, geom, row_ptr);   // next chunk's edges, in flight meanwhile
        if constexpr (BF) chunk_w_gemm_bf16<H, true>(D, L, smem, W3T_h);
        else chunk_w_gemm_f32<H>(D, L, smem, W3);
        switch (D.kind) {
            case 0: tp_fwd_chunk<H, LMAX, 0, WT>(D, ne, s_w, smem + L.G, s_src, s_dst, s_first, x, m); break;
            case 1: tp_fwd_chunk<H, LMAX, 1, WT>(D, ne, s_w, smem + L.G, s_src, s_dst, s_first, x, m); break;
            case 2: tp_fwd_chunk<H, LMAX, 2, WT>(D, ne, s_w, smem + L.G, s_src, s_dst, s_first, x, m); break;
            default: tp_fwd_chunk<H, LMAX, 3, WT>(D, ne, s_w, smem + L.G, s_src, s_dst, s_first, x, m); break;
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
size_t conv_smem_bytes(const ConvDesc& D, int H, bool bwd) { return smem_bytes(D, H, bwd, false); }

sevennet_status conv_configure_fwd(int H, size_t need) {
    static size_t granted[2][2] = {{0, 0}, {0, 0}};
    const int hi = H == 64 ? 1 : 0;
    if (H == 64) {
        SN_TRY(conv_set_smem((const void*)conv_fwd_kernel<64, false, 1>, need, &granted[hi][0]));
        SN_TRY(conv_set_smem((const void*)conv_fwd_kernel<64, true, 1>, need, &granted[hi][0]));
        SN_TRY(conv_set_smem((const void*)conv_fwd_kernel<64, false, 2>, need, &granted[hi][0]));
        SN_TRY(conv_set_smem((const void*)conv_fwd_kernel<64, true, 2>, need, &granted[hi][0]));
        SN_TRY(conv_set_smem((const void*)conv_fwd_kernel<64, false, 3>, need, &granted[hi][1]));
        SN_TRY(conv_set_smem((const void*)conv_fwd_kernel<64, true, 3>, need, &granted[hi][1]));
    } else if (H == 32) {
        SN_TRY(conv_set_smem((const void*)conv_fwd_kernel<32, false, 1>, need, &granted[hi][0]));
        SN_TRY(conv_set_smem((const void*)conv_fwd_kernel<32, true, 1>, need, &granted[hi][0]));
        SN_TRY(conv_set_smem((const void*)conv_fwd_kernel<32, false, 2>, need, &granted[hi][0]));
        SN_TRY(conv_set_smem((const void*)conv_fwd_kernel<32, true, 2>, need, &granted[hi][0]));
    } else {
        set_error("radial MLP hidden width must be 32 or 64");
        return SEVENNET_EINVAL;
    }
    return SEVENNET_OK;
}

void launch_conv_fwd(const LayerDev& L, int H, sevennet_precision prec, int64_t n_atoms,
                     int64_t n_edges, const int* row_ptr, const int* dst, const int* src,
                     const float4* geom, const float* x, float* m, cudaStream_t st, int* flags) {
    const int lm = L.conv.lmax;
    const bool bf = prec == SEVENNET_BF16;
    // BF16: the tensor-core contraction (conv_fwd_tc.cu) where the block allows
    // it; its bulk copies of the x rows want 16-byte aligned rows
    if (bf && L.conv.tc_ok && (reinterpret_cast<uintptr_t>(x) & 15) == 0) {
        launch_conv_fwd_tc(L, H, n_atoms, n_edges, row_ptr, dst, src, geom, x, m, flags, st);
        return;
    }
    const int grid = conv_grid(n_atoms, conv_ctas_per_sm(lm));
    const size_t sm = smem_bytes(L.conv, H, false, prec == SEVENNET_BF16);
#define SN_LF(HH, BB, LL) conv_fwd_kernel<HH, BB, LL><<<grid, CONV_THREADS, sm, st>>>(             \
        L.conv, L.mlp0, L.mlp1, L.mlp2, L.mlp2h, L.mlp1Th, (int)n_atoms, (int)n_edges, row_ptr, dst, src, geom, x, m)
    if (H == 64) {
        if (bf) { if (lm == 3) SN_LF(64, true, 3); else if (lm == 2) SN_LF(64, true, 2); else SN_LF(64, true, 1); }
        else    { if (lm == 3) SN_LF(64, false, 3); else if (lm == 2) SN_LF(64, false, 2); else SN_LF(64, false, 1); }
    } else {
        if (bf) { if (lm == 2) SN_LF(32, true, 2); else SN_LF(32, true, 1); }
        else    { if (lm == 2) SN_LF(32, false, 2); else SN_LF(32, false, 1); }
    }
#undef SN_LF
}

}  // namespace sn
