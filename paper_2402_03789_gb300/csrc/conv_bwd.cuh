// Adjoint of the tensor-product convolution (Eqs. 5 and 8): given dE/dm,
// dE/dx of the senders and dE/dd of every edge through the tensor product, the
// radial MLP and the edge embedding.  Shared phases live in conv_common.cuh;
// conv_bwd.cu instantiates the per-edge kernel, conv_bwd_pair.cu the one over
// unordered pairs.
#pragma once
#include "conv_common.cuh"

namespace sn {

// ------------------------------------------------------------- adjoint
// One path of one edge for CPL channels per lane (channels u0 + 32 k): the
// G matrix and the address arithmetic serve all of them.
template <int L1, int L2, int L3, int CPL>
__device__ __forceinline__ void tp_bwd_path(const PathDesc& P, int u0, int e, int v, const float (*xv)[2 * L1 + 1],
                                            float (*gx)[2 * L1 + 1], float* gY, float* s_w, int Wpad,
                                            const float* s_G, int nG,
                                            const float* __restrict__ gm, int m_dim) {
    constexpr int N1 = 2 * L1 + 1, N3 = 2 * L3 + 1;
    float* wr = s_w + e * Wpad + P.col0 + u0;
    const float* gmr = gm + (size_t)v * m_dim + P.m_off + P.m_ch0 + u0;
    float g[CPL][N3];
#pragma unroll
    for (int k = 0; k < CPL; ++k)
#pragma unroll
        for (int c = 0; c < N3; ++c) g[k][c] = __ldg(gmr + c * P.m_mul + 32 * k);
    float G[((N1 * N3 + 3) / 4) * 4];
    load_G<N1 * N3>(s_G + e * nG + P.g_off, G);
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        const float wv = wr[32 * k];
        float gw = 0.0f;
        float wx[N1];
#pragma unroll
        for (int a = 0; a < N1; ++a) {
            float tt = 0.0f;
#pragma unroll
            for (int c = 0; c < N3; ++c) tt = fmaf(G[a * N3 + c], g[k][c], tt);
            gw = fmaf(xv[k][a], tt, gw);
            gx[k][a] = fmaf(wv, tt, gx[k][a]);
            wx[a] = wv * xv[k][a];
        }
        wr[32 * k] = gw;             // dE/dw replaces w (same thread, same slot)
        CG<L1, L2, L3>::gY(wx, g[k], gY + L2 * L2);
    }
}

// Fixed-point add of one dE/dx contribution (order-independent sums); the
// conversion after the kernel reports a sum that received the sentinel.
__device__ __forceinline__ void gx_fixed_add(unsigned long long* p, float v) {
    const long long q = fabsf(v) < GX_LIMIT ? __float2ll_rn(v * GX_SCALE) : GX_SENTINEL;   // exact scaling by 2^36
    atomicAdd(p, (unsigned long long)q);
}

// All paths of one input irrep l1 for one edge, CPL channels per lane: the
// channel loads, the path descriptors and the CG code resolve at compile time.
template <int L1, int LMAX, int KIND, int CPL>
__device__ __forceinline__ void tp_bwd_block(const ConvDesc& D, int u0, int e, int v, int sidx, float* gY,
                                             float* s_w, const float* s_G, const float* __restrict__ x,
                                             const float* __restrict__ gm, unsigned long long* __restrict__ gxo) {
    using BP = BlockPaths<L1, LMAX, KIND>;
    constexpr int N1 = 2 * L1 + 1;
    const int mul = D.mul_in[L1];
    const float* xr = x + (size_t)sidx * D.x_dim + D.x_off[L1] + u0;
    unsigned long long* gxr = gxo ? gxo + (size_t)sidx * D.x_dim + D.x_off[L1] + u0 : nullptr;
    float xv[CPL][N1], gx[CPL][N1];
#pragma unroll
    for (int k = 0; k < CPL; ++k)
#pragma unroll
        for (int a = 0; a < N1; ++a) {
            xv[k][a] = __ldg(xr + a * mul + 32 * k);
            gx[k][a] = 0.0f;
        }
    static_for<BP::list.n>([&](auto I) {
        constexpr int i = decltype(I)::value;
        tp_bwd_path<L1, BP::list.l2[i], BP::list.l3[i], CPL>(D.paths[BP::begin + i], u0, e, v, xv, gx, gY,
                                                             s_w, D.Wpad, s_G, D.nG, gm, D.m_dim);
    });
    if (gxr) {                                   // null: the block's dE/dx is not needed
#pragma unroll
        for (int k = 0; k < CPL; ++k)
#pragma unroll
            for (int a = 0; a < N1; ++a) gx_fixed_add(gxr + a * mul + 32 * k, gx[k][a]);
    }
}

template <int L1, int LMAX, int KIND, int MAXC>
__device__ __forceinline__ void tp_bwd_l1(const ConvDesc& D, int lane, int e, int v, int sidx,
                                          float* gY, float* s_w, const float* s_G,
                                          const float* __restrict__ x,
                                          const float* __restrict__ gm, unsigned long long* __restrict__ gxo) {
    if constexpr (BlockPaths<L1, LMAX, KIND>::list.n > 0) {
        const int mul = D.mul_in[L1];
        for (int ub = 0; ub < mul;) {
            const int left = (mul - ub) / 32;
            if (MAXC >= 4 && left >= 4) {
                tp_bwd_block<L1, LMAX, KIND, (MAXC >= 4 ? 4 : 1)>(D, ub + lane, e, v, sidx, gY, s_w, s_G, x, gm, gxo);
                ub += 128;
            } else if (MAXC >= 2 && left >= 2) {
                tp_bwd_block<L1, LMAX, KIND, (MAXC >= 2 ? 2 : 1)>(D, ub + lane, e, v, sidx, gY, s_w, s_G, x, gm, gxo);
                ub += 64;
            } else {
                tp_bwd_block<L1, LMAX, KIND, 1>(D, ub + lane, e, v, sidx, gY, s_w, s_G, x, gm, gxo);
                ub += 32;
            }
        }
    }
}

// Phase E of the adjoint for every edge of the chunk (warp per edge).
template <int LMAX, int KIND, int MAXC>
__device__ __forceinline__ void tp_bwd_chunk(const ConvDesc& D, int ne, const int* s_dst, const int* s_src,
                                             float* s_w, const float* s_G, float* s_gY,
                                             const float* __restrict__ x, const float* __restrict__ gm,
                                             unsigned long long* __restrict__ gx) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int e = warp; e < ne; e += CONV_WARPS) {
        const int v = s_dst[e], sidx = s_src[e];
        constexpr int NYS = LMAX >= 3 ? 16 : 9;
        float gY[NYS];
#pragma unroll
        for (int i = 0; i < NYS; ++i) gY[i] = 0.0f;
        tp_bwd_l1<0, LMAX, KIND, MAXC>(D, lane, e, v, sidx, gY, s_w, s_G, x, gm, gx);
        tp_bwd_l1<1, LMAX, KIND, MAXC>(D, lane, e, v, sidx, gY, s_w, s_G, x, gm, gx);
        if constexpr (LMAX >= 2) tp_bwd_l1<2, LMAX, KIND, MAXC>(D, lane, e, v, sidx, gY, s_w, s_G, x, gm, gx);
        if constexpr (LMAX >= 3) tp_bwd_l1<3, LMAX, KIND, MAXC>(D, lane, e, v, sidx, gY, s_w, s_G, x, gm, gx);
        constexpr int NY = (LMAX + 1) * (LMAX + 1);
#pragma unroll
        for (int i = 0; i < NY; ++i) gY[i] = warp_sum(gY[i]);
        if (lane < NYS) {
            float val = 0.0f;
#pragma unroll
            for (int i = 0; i < NY; ++i) if (lane == i) val = gY[i];
            s_gY[e * y_stride<LMAX>() + lane] = val;
        }
    }
}

// ------------------------------------------------------------- unordered pairs
// An edge e (receiver v, sender w, d = r_w + S cell - r_v) and its reverse
// (receiver w, sender v, -d) share the radial weights w_e, which depend on |d|
// only, and Y_l(-d/r) = (-1)^l Y_l(d/r), so G of the reverse is (-1)^l2 G.  The
// pair kernel runs the radial MLP, the G matrices and their adjoints once per
// pair and the tensor product once per direction: direction a is e itself,
// direction b takes dE/dm of w times (-1)^l2 and x of v, which gives the
// reverse edge's products expressed through Y(d/r).  dE/dw, and dE/dY w.r.t.
// Y(d/r), are the sums over both directions.
template <int L1, int L2, int L3, int CPL>
__device__ __forceinline__ void tp_bwd_path_pair(const PathDesc& P, int u0, int e, int v, int w,
                                                 const float (*xa)[2 * L1 + 1], const float (*xb)[2 * L1 + 1],
                                                 float (*gxa)[2 * L1 + 1], float (*gxb)[2 * L1 + 1], float* gY,
                                                 float* s_w, int Wpad, const float* s_G, int nG,
                                                 const float* __restrict__ gm, int m_dim) {
    constexpr int N1 = 2 * L1 + 1, N3 = 2 * L3 + 1;
    constexpr float sb = (L2 & 1) ? -1.0f : 1.0f;
    float* wr = s_w + e * Wpad + P.col0 + u0;
    const float* gma = gm + (size_t)v * m_dim + P.m_off + P.m_ch0 + u0;
    const float* gmb = gm + (size_t)w * m_dim + P.m_off + P.m_ch0 + u0;
    float ga[CPL][N3], gb[CPL][N3];
#pragma unroll
    for (int k = 0; k < CPL; ++k)
#pragma unroll
        for (int c = 0; c < N3; ++c) {
            ga[k][c] = __ldg(gma + c * P.m_mul + 32 * k);
            gb[k][c] = sb * __ldg(gmb + c * P.m_mul + 32 * k);
        }
    float G[((N1 * N3 + 3) / 4) * 4];
    load_G<N1 * N3>(s_G + e * nG + P.g_off, G);
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        const float wv = wr[32 * k];
        float gw = 0.0f;
        float wx[N1];
#pragma unroll
        for (int a = 0; a < N1; ++a) {
            float tt = 0.0f;
#pragma unroll
            for (int c = 0; c < N3; ++c) tt = fmaf(G[a * N3 + c], ga[k][c], tt);
            gw = fmaf(xa[k][a], tt, gw);
            gxa[k][a] = fmaf(wv, tt, gxa[k][a]);
            wx[a] = wv * xa[k][a];
        }
        CG<L1, L2, L3>::gY(wx, ga[k], gY + L2 * L2);
#pragma unroll
        for (int a = 0; a < N1; ++a) {
            float tt = 0.0f;
#pragma unroll
            for (int c = 0; c < N3; ++c) tt = fmaf(G[a * N3 + c], gb[k][c], tt);
            gw = fmaf(xb[k][a], tt, gw);
            gxb[k][a] = fmaf(wv, tt, gxb[k][a]);
            wx[a] = wv * xb[k][a];
        }
        CG<L1, L2, L3>::gY(wx, gb[k], gY + L2 * L2);
        wr[32 * k] = gw;             // dE/dw of the pair replaces w
    }
}

template <int L1, int LMAX, int KIND, int CPL>
__device__ __forceinline__ void tp_bwd_block_pair(const ConvDesc& D, int u0, int e, int v, int w, float* gY,
                                                  float* s_w, const float* s_G, const float* __restrict__ x,
                                                  const float* __restrict__ gm,
                                                  unsigned long long* __restrict__ gxo) {
    using BP = BlockPaths<L1, LMAX, KIND>;
    constexpr int N1 = 2 * L1 + 1;
    const int mul = D.mul_in[L1];
    const float* xra = x + (size_t)w * D.x_dim + D.x_off[L1] + u0;     // direction a: sender w
    const float* xrb = x + (size_t)v * D.x_dim + D.x_off[L1] + u0;     // direction b: sender v
    float xa[CPL][N1], xb[CPL][N1], gxa[CPL][N1], gxb[CPL][N1];
#pragma unroll
    for (int k = 0; k < CPL; ++k)
#pragma unroll
        for (int a = 0; a < N1; ++a) {
            xa[k][a] = __ldg(xra + a * mul + 32 * k);
            xb[k][a] = __ldg(xrb + a * mul + 32 * k);
            gxa[k][a] = 0.0f;
            gxb[k][a] = 0.0f;
        }
    static_for<BP::list.n>([&](auto I) {
        constexpr int i = decltype(I)::value;
        tp_bwd_path_pair<L1, BP::list.l2[i], BP::list.l3[i], CPL>(D.paths[BP::begin + i], u0, e, v, w, xa, xb,
                                                                  gxa, gxb, gY, s_w, D.Wpad, s_G, D.nG, gm,
                                                                  D.m_dim);
    });
    if (gxo) {                                   // null: the block's dE/dx is not needed
        unsigned long long* ra = gxo + (size_t)w * D.x_dim + D.x_off[L1] + u0;
        unsigned long long* rb = gxo + (size_t)v * D.x_dim + D.x_off[L1] + u0;
#pragma unroll
        for (int k = 0; k < CPL; ++k)
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                gx_fixed_add(ra + a * mul + 32 * k, gxa[k][a]);
                gx_fixed_add(rb + a * mul + 32 * k, gxb[k][a]);
            }
    }
}

template <int L1, int LMAX, int KIND, int MAXC>
__device__ __forceinline__ void tp_bwd_l1_pair(const ConvDesc& D, int lane, int e, int v, int w, float* gY,
                                               float* s_w, const float* s_G, const float* __restrict__ x,
                                               const float* __restrict__ gm, unsigned long long* __restrict__ gxo) {
    if constexpr (BlockPaths<L1, LMAX, KIND>::list.n > 0) {
        const int mul = D.mul_in[L1];
        for (int ub = 0; ub < mul;) {
            const int left = (mul - ub) / 32;
            if (MAXC >= 2 && left >= 2) {
                tp_bwd_block_pair<L1, LMAX, KIND, (MAXC >= 2 ? 2 : 1)>(D, ub + lane, e, v, w, gY, s_w, s_G, x, gm,
                                                                       gxo);
                ub += 64;
            } else {
                tp_bwd_block_pair<L1, LMAX, KIND, 1>(D, ub + lane, e, v, w, gY, s_w, s_G, x, gm, gxo);
                ub += 32;
            }
        }
    }
}

// Phase E of the pair kernel: a warp per pair (slot e: receiver v = s_dst[e],
// sender w = s_src[e]).
template <int LMAX, int KIND, int MAXC>
__device__ __forceinline__ void tp_bwd_chunk_pair(const ConvDesc& D, int ne, const int* s_dst, const int* s_src,
                                                  float* s_w, const float* s_G, float* s_gY,
                                                  const float* __restrict__ x, const float* __restrict__ gm,
                                                  unsigned long long* __restrict__ gx) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int e = warp; e < ne; e += CONV_WARPS) {
        const int v = s_dst[e], w = s_src[e];
        constexpr int NYS = LMAX >= 3 ? 16 : 9;
        float gY[NYS];
#pragma unroll
        for (int i = 0; i < NYS; ++i) gY[i] = 0.0f;
        // l1 = 0 (one component per channel) takes two channels per lane; the
        // others one (two spill; measured 0.31 ms faster than one everywhere)
        tp_bwd_l1_pair<0, LMAX, KIND, 2 * MAXC>(D, lane, e, v, w, gY, s_w, s_G, x, gm, gx);
        tp_bwd_l1_pair<1, LMAX, KIND, MAXC>(D, lane, e, v, w, gY, s_w, s_G, x, gm, gx);
        if constexpr (LMAX >= 2) tp_bwd_l1_pair<2, LMAX, KIND, MAXC>(D, lane, e, v, w, gY, s_w, s_G, x, gm, gx);
        if constexpr (LMAX >= 3) tp_bwd_l1_pair<3, LMAX, KIND, MAXC>(D, lane, e, v, w, gY, s_w, s_G, x, gm, gx);
        constexpr int NY = (LMAX + 1) * (LMAX + 1);
#pragma unroll
        for (int i = 0; i < NY; ++i) gY[i] = warp_sum(gY[i]);
        if (lane < NYS) {
            float val = 0.0f;
#pragma unroll
            for (int i = 0; i < NY; ++i) if (lane == i) val = gY[i];
            s_gY[e * y_stride<LMAX>() + lane] = val;
        }
    }
}

// PAIR = false: one unit per edge, records (dst, src, geom) indexed by edge.
// PAIR = true: one unit per unordered pair, records in pair order and eidx[]
// the pair's edge, which receives the pair's whole dE/dd (its reverse keeps 0:
// forces and virials use dE/dd_e - dE/dd_rev(e) only).  *count is the number of
// units (read on the device).
template <int H, bool BF, int LMAX, bool PAIR>
__global__ void __launch_bounds__(CONV_THREADS, conv_ctas_per_sm(LMAX))
conv_bwd_kernel(const ConvDesc D, const float* __restrict__ W1, const float* __restrict__ W2,
                const float* __restrict__ W2T, const float* __restrict__ W3, const float* __restrict__ W3T,
                const __nv_bfloat16* __restrict__ W3T_h, const __nv_bfloat16* __restrict__ W3_h,
                const __nv_bfloat16* __restrict__ W2T_h, const __nv_bfloat16* __restrict__ W2_h,
                int tile_units, const int* __restrict__ count, const int* __restrict__ dst,
                const int* __restrict__ src, const float4* __restrict__ geom, const int* __restrict__ eidx,
                const float* __restrict__ x, const float* __restrict__ gm,
                unsigned long long* __restrict__ gx, float* __restrict__ gd) {
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    const ConvSmem L = conv_smem_layout(D.Wpad, D.WpadB, H, D.nG, D.ys, true, BF);
    // One tile of tile_units units (edges or pairs) per CTA, CTA k taking tile k:
    // every output is per unit (dE/dd) or an order-independent sum (dE/dx), so
    // tiles need not follow receiver boundaries.  CTAs start in index order as earlier ones
    // finish, so the resident CTAs sweep one narrow window of receivers at a
    // time, and the senders of that window (atoms near it in the cell-list
    // order), their x rows and dE/dx sums, stay in L2.
    __shared__ int s_range[2];
    if (threadIdx.x == 0) {
        const long long n_e = *count, lo = (long long)blockIdx.x * tile_units;
        s_range[0] = (int)min(lo, n_e);
        s_range[1] = (int)min(lo + tile_units, n_e);
    }
    __syncthreads();
    const int E0 = s_range[0], E1 = s_range[1];
    if (E0 >= E1) return;                        // beyond the device-side unit count
    const int t = threadIdx.x, warp = t >> 5;
    const int* s_src = reinterpret_cast<const int*>(smem + L.src);
    const int* s_dst = reinterpret_cast<const int*>(smem + L.dst);
    float* s_w = smem + L.w;
    float* s_gY = smem + L.gY;
    load_W1<H>(D, L, smem, W1);
    float* s_gdp = smem + L.gdp;
    // The next chunk's edge records are copied to shared memory asynchronously
    // (thread e < EC copies edge e), so no registers hold them across a chunk.
    __shared__ float4 s_ngeo[EC];
    __shared__ int s_nsrc[EC], s_ndst[EC], s_ne[PAIR ? EC : 1], s_ecur[PAIR ? EC : 1];
    auto stage = [&](int c) {
        if (t < EC && c + t < E1) {
            cp_async4(reinterpret_cast<float*>(s_nsrc + t), reinterpret_cast<const float*>(src + c + t));
            cp_async4(reinterpret_cast<float*>(s_ndst + t), reinterpret_cast<const float*>(dst + c + t));
            cp_async16(s_ngeo + t, geom + c + t);
            if constexpr (PAIR) cp_async4(reinterpret_cast<float*>(s_ne + t), reinterpret_cast<const float*>(eidx + c + t));
        }
    };
    stage(E0);
    cp_async_commit();
    cp_async_wait_all();
    for (int c0 = E0; c0 < E1; c0 += EC) {
        const int ne = min(EC, E1 - c0);
        __syncthreads();
        EdgePrefetch cur;
        if (t < ne) {
            cur.src = s_nsrc[t];
            cur.dst = s_ndst[t];
            cur.geom = s_ngeo[t];
            if constexpr (PAIR) s_ecur[t] = s_ne[t];      // published by the prologue's barrier
        }
        chunk_prologue<H, BF, LMAX>(D, L, smem, c0, ne, cur, W2, W2T_h);
        stage(c0 + EC);        // lands by the wait before phase G
        // dE/dd of the blocks done so far, copied to shared memory for phase G
        if (t < 3 * ne) {
            if constexpr (PAIR) cp_async4(s_gdp + t, gd + (size_t)s_ecur[t / 3] * 3 + t % 3);
            else cp_async4(s_gdp + t, gd + (size_t)c0 * 3 + t);
        }
        cp_async_commit();
        if constexpr (BF) chunk_w_gemm_bf16<H, false>(D, L, smem, W3T_h);
        else chunk_w_gemm_f32<H>(D, L, smem, W3);
        // E: per-edge (or per-pair) adjoint of the tensor product (path lists fixed per
        // block kind); the H = 32 kernels (small models) take one channel per lane
        constexpr int MAXC = H == 64 ? 2 : 1;
        if constexpr (PAIR) {      // one channel per lane for l1 >= 1: two directions' operands in registers
            switch (D.kind) {
                case 0: tp_bwd_chunk_pair<LMAX, 0, 1>(D, ne, s_dst, s_src, s_w, smem + L.G, s_gY, x, gm, gx); break;
                case 1: tp_bwd_chunk_pair<LMAX, 1, 1>(D, ne, s_dst, s_src, s_w, smem + L.G, s_gY, x, gm, gx); break;
                case 2: tp_bwd_chunk_pair<LMAX, 2, 1>(D, ne, s_dst, s_src, s_w, smem + L.G, s_gY, x, gm, gx); break;
                default: tp_bwd_chunk_pair<LMAX, 3, 1>(D, ne, s_dst, s_src, s_w, smem + L.G, s_gY, x, gm, gx); break;
            }
        } else {
            switch (D.kind) {
                case 0: tp_bwd_chunk<LMAX, 0, MAXC>(D, ne, s_dst, s_src, s_w, smem + L.G, s_gY, x, gm, gx); break;
                case 1: tp_bwd_chunk<LMAX, 1, MAXC>(D, ne, s_dst, s_src, s_w, smem + L.G, s_gY, x, gm, gx); break;
                case 2: tp_bwd_chunk<LMAX, 2, MAXC>(D, ne, s_dst, s_src, s_w, smem + L.G, s_gY, x, gm, gx); break;
                default: tp_bwd_chunk<LMAX, 3, MAXC>(D, ne, s_dst, s_src, s_w, smem + L.G, s_gY, x, gm, gx); break;
            }
        }
        // F: dE/dH2 = dE/dw @ W3^T
        if constexpr (BF) chunk_gw_gemm_bf16<H, PAIR>(D, L, smem, W3_h);
        else chunk_gw_gemm_f32<H>(D, L, smem, W3T);
        // MLP adjoint: gA2 = gH2 * silu'(A2); gH1 = gA2 @ W2^T; gA1 = gH1 * silu'(A1); gB = gA1 @ W1^T
        float* s_gH = smem + L.gH;
        float* s_A1 = smem + L.A1;
        float* s_A2 = smem + L.A2;
        for (int i = t; i < H * EC; i += CONV_THREADS) s_gH[i] *= dsiluf_(s_A2[i]);
        __syncthreads();
        if constexpr (BF) {   // gA1 = (gA2 @ W2^T) * silu'(A1) on tensor cores, stored over A2
            const int lane = t & 31, g = lane >> 2, tq = lane & 3;
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            const int nt = warp;
            if (nt < H / 8) {
                HiddenB<H> hb;
                hidden_load<H>(W2_h, nt, hb);
                hidden_mma<H, PAIR>(s_gH, hb, c);
            }
            __syncthreads();       // every read of A2 (the silu' above) is done
            if (nt < H / 8) {
                const int k = nt * 8 + 2 * tq;
                const int o[4] = {hk<H>(k, g), hk<H>(k + 1, g), hk<H>(k, g + 8), hk<H>(k + 1, g + 8)};
#pragma unroll
                for (int q = 0; q < 4; ++q) s_A2[o[q]] = c[q] * dsiluf_(s_A1[o[q]]);
            }
        } else {   // gA1 = (gA2 @ W2^T) * silu'(A1), stored over A2; W2T[j][k] = W2[k][j]
            float ga[(H / 4) * EC / CONV_THREADS > 0 ? (H / 4) * EC / CONV_THREADS : 1][4];
            int nq = 0;
            for (int idx = t; idx < (H / 4) * EC; idx += CONV_THREADS, ++nq) {
                const int kq = idx / EC, e = idx % EC;
                float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll 8
                for (int j = 0; j < H; ++j) {
                    const float4 b = __ldg(reinterpret_cast<const float4*>(W2T + j * H) + kq);
                    const float a = s_gH[hk<H>(j, e)];
                    a0 = fmaf(a, b.x, a0);
                    a1 = fmaf(a, b.y, a1);
                    a2 = fmaf(a, b.z, a2);
                    a3 = fmaf(a, b.w, a3);
                }
                ga[nq][0] = a0; ga[nq][1] = a1; ga[nq][2] = a2; ga[nq][3] = a3;
            }
            __syncthreads();       // every read of A2 (the silu' above) is done
            nq = 0;
            for (int idx = t; idx < (H / 4) * EC; idx += CONV_THREADS, ++nq) {
                const int kq = idx / EC, e = idx % EC;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int o = hk<H>(4 * kq + q, e);
                    s_A2[o] = ga[nq][q] * dsiluf_(s_A1[o]);
                }
            }
        }
        __syncthreads();
        float* s_gB = smem + L.stage;              // [NB][EC]
        for (int i = t; i < D.n_basis * EC; i += CONV_THREADS) {
            const int n = i / EC, e = i % EC;
            float a = 0.0f;
#pragma unroll 8
            for (int k = 0; k < H; ++k) a = fmaf(s_A2[hk<H>(k, e)], smem[L.W1 + n * H + k], a);
            s_gB[i] = a;
        }
        cp_async_wait_all();
        __syncthreads();
        // G: dE/dd = (dE/dr) u + (I - u u^T) dE/du / r
        if (t < ne) {
            const float4 g = reinterpret_cast<const float4*>(smem + L.geo)[t];
            const float r = g.w, inv = 1.0f / r;
            const float ux = g.x * inv, uy = g.y * inv, uz = g.z * inv;
            float env, denv;
            envelope(D, r / D.r_cut, env, denv);
            denv /= D.r_cut;
            const float th = 3.14159265358979f * r / D.r_cut;
            const float dth = 3.14159265358979f / D.r_cut;
            float s1, c1;
            sincosf(th, &s1, &c1);
            float sm = 0.0f, sn = s1, cm = 1.0f, cn = c1;
            const float k2 = 2.0f / D.r_cut;
            float dEdr = 0.0f;
            for (int n = 0; n < D.n_basis; ++n) {
                const float nn = (float)(n + 1);
                const float f = k2 * sn * inv;
                const float df = k2 * (nn * dth * cn * inv - sn * inv * inv);
                dEdr = fmaf(s_gB[n * EC + t], df * env + f * denv, dEdr);
                const float ns = 2.0f * c1 * sn - sm;
                const float nc = 2.0f * c1 * cn - cm;
                sm = sn; sn = ns; cm = cn; cn = nc;
            }
            const float* gy = s_gY + t * y_stride<LMAX>();
            const float s3 = 1.7320508075688772f, s15 = 3.872983346207417f, s5 = 2.23606797749979f;
            float gux = s3 * gy[3], guy = s3 * gy[1], guz = s3 * gy[2];
            if (D.lmax >= 2) {
                gux += s15 * (uy * gy[4] + uz * gy[7] + ux * gy[8]);
                guy += s15 * (ux * gy[4] + uz * gy[5] - uy * gy[8]);
                guz += s15 * (uy * gy[5] + ux * gy[7]) + 3.0f * s5 * uz * gy[6];
            }
            if constexpr (LMAX >= 3) {   // gradients of the degree-3 polynomials (projected below)
                const float a3 = 2.0916500663351889f, b3 = 10.246950765959598f;
                const float c3 = 1.6201851746019651f, d3 = 1.3228756555322954f;
                const float zz5 = 5.0f * uz * uz - 1.0f;
                gux += gy[9] * 6.0f * a3 * ux * uy + gy[10] * b3 * uy * uz + gy[13] * c3 * zz5 +
                       gy[14] * b3 * ux * uz + gy[15] * 3.0f * a3 * (ux * ux - uy * uy);
                guy += gy[9] * 3.0f * a3 * (ux * ux - uy * uy) + gy[10] * b3 * ux * uz + gy[11] * c3 * zz5 -
                       gy[14] * b3 * uy * uz - gy[15] * 6.0f * a3 * ux * uy;
                guz += gy[10] * b3 * ux * uy + gy[11] * 10.0f * c3 * uy * uz +
                       gy[12] * d3 * (15.0f * uz * uz - 3.0f) + gy[13] * 10.0f * c3 * ux * uz +
                       gy[14] * 0.5f * b3 * (ux * ux - uy * uy);
            }
            const float dot = gux * ux + guy * uy + guz * uz;
            float* o = gd + (size_t)(PAIR ? s_ecur[t] : c0 + t) * 3;
            o[0] = s_gdp[3 * t] + dEdr * ux + (gux - dot * ux) * inv;
            o[1] = s_gdp[3 * t + 1] + dEdr * uy + (guy - dot * uy) * inv;
            o[2] = s_gdp[3 * t + 2] + dEdr * uz + (guz - dot * uz) * inv;
        }
    }
}

// ------------------------------------------------------------- host side
template <bool PAIR>
sevennet_status conv_configure_bwd_mode(int H, size_t need) {
    static size_t granted[2][2] = {{0, 0}, {0, 0}};
    const int hi = H == 64 ? 1 : 0;
    if (H == 64) {
        SN_TRY(conv_set_smem((const void*)conv_bwd_kernel<64, false, 1, PAIR>, need, &granted[hi][0]));
        SN_TRY(conv_set_smem((const void*)conv_bwd_kernel<64, true, 1, PAIR>, need, &granted[hi][0]));
        SN_TRY(conv_set_smem((const void*)conv_bwd_kernel<64, false, 2, PAIR>, need, &granted[hi][0]));
        SN_TRY(conv_set_smem((const void*)conv_bwd_kernel<64, true, 2, PAIR>, need, &granted[hi][0]));
        SN_TRY(conv_set_smem((const void*)conv_bwd_kernel<64, false, 3, PAIR>, need, &granted[hi][1]));
        SN_TRY(conv_set_smem((const void*)conv_bwd_kernel<64, true, 3, PAIR>, need, &granted[hi][1]));
    } else if (H == 32) {
        SN_TRY(conv_set_smem((const void*)conv_bwd_kernel<32, false, 1, PAIR>, need, &granted[hi][0]));
        SN_TRY(conv_set_smem((const void*)conv_bwd_kernel<32, true, 1, PAIR>, need, &granted[hi][0]));
        SN_TRY(conv_set_smem((const void*)conv_bwd_kernel<32, false, 2, PAIR>, need, &granted[hi][0]));
        SN_TRY(conv_set_smem((const void*)conv_bwd_kernel<32, true, 2, PAIR>, need, &granted[hi][0]));
    } else {
        set_error("radial MLP hidden width must be 32 or 64");
        return SEVENNET_EINVAL;
    }
    return SEVENNET_OK;
}

// bound: an upper bound on the number of units (the count itself is *count, on
// the device).  Tiles of 1..4 chunks, at least about 8 waves of tiles where the
// input allows (4 measured fastest on the 24,000-atom cell: 2 and 8 were slower).
template <bool PAIR>
void conv_bwd_dispatch(const LayerDev& L, int H, bool bf, int64_t bound, const int* count, const int* dst,
                       const int* src, const float4* geom, const int* eidx, const float* x, const float* gm,
                       unsigned long long* gxq, float* gd, cudaStream_t st) {
    const int lm = L.conv.lmax;
    bound = std::max<int64_t>(bound, 0);
    const int64_t wave = (int64_t)conv_grid(INT64_MAX, conv_ctas_per_sm(lm));
    const int tile = EC * (int)std::min<int64_t>(4, std::max<int64_t>(1, bound / (EC * 8 * wave)));
    const int grid = (int)std::max<int64_t>(1, (bound + tile - 1) / tile);
    const size_t sm = smem_bytes(L.conv, H, true, bf);
#define SN_LB(HH, BB, LL) conv_bwd_kernel<HH, BB, LL, PAIR><<<grid, CONV_THREADS, sm, st>>>(           \
        L.conv, L.mlp0, L.mlp1, L.mlp1T, L.mlp2, L.mlp2T, L.mlp2h, L.mlp2Th, L.mlp1Th, L.mlp1h,       \
        tile, count, dst, src, geom, eidx, x, gm, gxq, gd)
    if (H == 64) {
        if (bf) { if (lm == 3) SN_LB(64, true, 3); else if (lm == 2) SN_LB(64, true, 2); else SN_LB(64, true, 1); }
        else    { if (lm == 3) SN_LB(64, false, 3); else if (lm == 2) SN_LB(64, false, 2); else SN_LB(64, false, 1); }
    } else {
        if (bf) { if (lm == 2) SN_LB(32, true, 2); else SN_LB(32, true, 1); }
        else    { if (lm == 2) SN_LB(32, false, 2); else SN_LB(32, false, 1); }
    }
#undef SN_LB
}

}  // namespace sn
