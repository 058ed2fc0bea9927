// Shared device code of the tensor-product convolution (forward: conv_fwd.cu,
// adjoint: conv_bwd.cu).
//
// Tensor-product convolution of one interaction block and its adjoint.
//
// Forward (paper Eq. 3, Figure 2b; SevenNet-0 details Sec. 5.1):
//   m_v[p][m3, u] = sum_{e into v} w_e[p, u] sum_{m1} x_src(e)[l1][m1, u] G_e^p[m1, m3]
//   G_e^p[m1, m3] = sum_{m2} C_p[m1, m2, m3] Y_l2(d_e)[m2],
//   w_e = MLP(Bessel(r_e) * envelope(r_e))  (the 1/avg_num_neigh factor is folded into
//   the last MLP weight matrix on the host).
// Adjoint (Eqs. 5-8): given g_m = dE/dm, each edge produces dE/dx_src (scattered
// to the sender as 64-bit fixed-point sums), dE/dw_e -> back through the
// MLP to dE/dr_e, and dE/dY_e; together dE/dd_e, accumulated over blocks.
//
// Forward: one CTA owns a contiguous range of receivers (balanced by edge
// count) and walks its edges, sorted by receiver, in chunks of EC edges.
// Adjoint: one CTA per tile of up to 4 chunks, tiles in edge order.  Per chunk:
//   A  geometry: r, unit vector, Y (l <= 2), Bessel basis x envelope  (FP32)
//   B  radial MLP hidden layers                                      (FFMA)
//   C  G matrices of every path for every edge of the chunk
//   D  w = H2 @ W3 for all W columns into shared memory              (FFMA)
//   E  forward: each warp owns 32-channel groups of paths and walks the edges,
//      keeping the running sum of the current receiver in registers and writing
//      it once when the receiver changes (segmented sum, no atomics);
//      adjoint: each warp owns edges and walks all paths of that edge.
#pragma once

#include "internal.h"
#include "cg_tables.cuh"

#include <utility>

namespace sn {

constexpr int KS = 8;         // k-slice of the W3 staging in phase D
constexpr int DCOLS = 512;    // columns per pass of phase D
constexpr int CS = 32;        // column slice of phase F (adjoint W3 product)

struct ConvSmem {
    int w, stage, A1, A2, H2, gH, G, Y, B, gY, src, dst, first, W1, geo, gdp, total;
};

__host__ __device__ inline int rup4(int x) { return (x + 3) & ~3; }

// Index of element (k, e) of an [H][EC] activation tile (EC = 16).  Rows k and
// k + 1 share one 32-word line, and the line is XOR-permuted in 8-word steps by
// t(k) = (4 k / H + k / 2) mod 4.  The MMA fragment loads (the four tq lanes
// read rows H/4 apart) and the accumulator stores (rows 2 tq, 2 tq + 1) then
// touch 32 distinct banks, and four consecutive e stay contiguous and aligned.
template <int H>
__device__ __forceinline__ int hk(int k, int e) {
    const int t = ((k * 4 / H) + (k >> 1)) & 3;
    return ((k >> 1) << 5) | ((((k & 1) << 4) | e) ^ (t << 3));
}

// Inverse of hk: the (k, e) stored at position i.
template <int H>
__device__ __forceinline__ void hk_inv(int i, int& k, int& e) {
    const int line = i >> 5;
    const int t = ((line * 8 / H) + line) & 3;         // 4 k / H with k = 2 line (H / 4 is even)
    const int p = (i & 31) ^ (t << 3);
    k = 2 * line + (p >> 4);
    e = p & 15;
}

// The staging region holds H1 and dE/dbasis on both paths, and the W3 slices of
// the FP32 phases D and F on the FP32 path only.  dE/dH2 (adjoint) reuses H2,
// which is dead once phase D has run.  The BF16 kernels stay under 97 KB so two
// CTAs leave about 60 KB of each SM's 256 KB to the L1 cache.
__host__ __device__ inline ConvSmem conv_smem_layout(int Wpad, int WpadB, int H, int nG, int ys, bool bwd, bool bf) {
    ConvSmem s;
    int o = 0;
    const int stage_bf = H * EC > MAX_NB * EC ? H * EC : MAX_NB * EC;
    const int stage_f32 = KS * DCOLS > 2 * CS * 64 ? KS * DCOLS : 2 * CS * 64;
    // [EC][row stride]: BF16 in the BF16 forward; the BF16 adjoint also keeps three
    // [H][EC] partials of phase F there
    const int w_bwd_bf = EC * Wpad > 3 * H * EC ? EC * Wpad : 3 * H * EC;
    s.w = o;     o += (bf && !bwd) ? EC * WpadB / 2 : (bf ? w_bwd_bf : EC * Wpad);
    s.stage = o; o += bf ? stage_bf : (stage_f32 > stage_bf ? stage_f32 : stage_bf);
    s.A1 = o;    o += H * EC;
    s.A2 = o;    o += H * EC;
    s.H2 = o;    o += H * EC;
    s.gH = s.H2;
    s.G = o;     o += rup4(EC * nG);
    s.Y = o;     o += EC * ys;
    s.B = o;     o += MAX_NB * EC;
    s.gY = o;    o += bwd ? EC * ys : 0;
    s.src = o;   o += EC;
    s.dst = o;   o += EC;
    s.first = o; o += EC;
    s.W1 = o;    o += MAX_NB * H;          // radial MLP input layer, loaded once per CTA
    s.geo = o;   o += 4 * EC;              // (d, r) of the chunk's edges
    s.gdp = o;   o += bwd ? 3 * EC : 0;    // dE/dd of earlier blocks, prefetched (adjoint)
    s.total = o;
    return s;
}

__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + expf(-x)); }
__device__ __forceinline__ float siluf_(float x) { return x * sigmoidf_(x); }
__device__ __forceinline__ float dsiluf_(float x) {
    float s = sigmoidf_(x);
    return s * (1.0f + x * (1.0f - s));
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Envelope u(x) and du/dx for x = r / r_c (polynomial cutoff of order p).
__device__ __forceinline__ void envelope(const ConvDesc& D, float xr, float& u, float& du) {
    if (xr >= 1.0f) { u = 0.0f; du = 0.0f; return; }
    float xp1 = 1.0f;                       // x^(p-1)
    for (int i = 0; i < D.poly_p - 1; ++i) xp1 *= xr;
    float xp = xp1 * xr, xp2 = xp * xr, xp3 = xp2 * xr;
    const float p = (float)D.poly_p;
    u = 1.0f - D.env_a * xp + D.env_b * xp2 - D.env_c * xp3;
    du = -D.env_a * p * xp1 + D.env_b * (p + 1.0f) * xp - D.env_c * (p + 2.0f) * xp2;
}

// Phase A: Y_l(d/r) (component normalised, m = -l..l) and the enveloped basis.
template <int LMAX>
__device__ __forceinline__ void edge_features(const ConvDesc& D, float4 g, float* Y, float* Bcol,
                                              int bstride) {
    const float r = g.w;
    const float inv = 1.0f / r;
    const float x = g.x * inv, y = g.y * inv, z = g.z * inv;
    const float s3 = 1.7320508075688772f, s15 = 3.872983346207417f, s5 = 2.23606797749979f;
    Y[0] = 1.0f;
    Y[1] = s3 * y; Y[2] = s3 * z; Y[3] = s3 * x;
    if (D.lmax >= 2) {
        Y[4] = s15 * x * y;
        Y[5] = s15 * y * z;
        Y[6] = 0.5f * s5 * (3.0f * z * z - 1.0f);
        Y[7] = s15 * x * z;
        Y[8] = 0.5f * s15 * (x * x - y * y);
    } else {
        Y[4] = Y[5] = Y[6] = Y[7] = Y[8] = 0.0f;
    }
    if constexpr (LMAX >= 3) {   // degree 3 (m = -3..3), the standard real harmonics times sqrt(4 pi)
        const float a3 = 2.0916500663351889f, b3 = 10.246950765959598f;    // sqrt(70)/4, sqrt(105)
        const float c3 = 1.6201851746019651f, d3 = 1.3228756555322954f;    // sqrt(42)/4, sqrt(7)/2
        const float zz5 = 5.0f * z * z;
        Y[9] = a3 * y * (3.0f * x * x - y * y);
        Y[10] = b3 * x * y * z;
        Y[11] = c3 * y * (zz5 - 1.0f);
        Y[12] = d3 * z * (zz5 - 3.0f);
        Y[13] = c3 * x * (zz5 - 1.0f);
        Y[14] = 0.5f * b3 * z * (x * x - y * y);
        Y[15] = a3 * x * (x * x - 3.0f * y * y);
    }
    float u, du;
    envelope(D, r / D.r_cut, u, du);
    const float th = 3.14159265358979f * r / D.r_cut;
    float s1, c1;
    sincosf(th, &s1, &c1);
    const float pref = 2.0f / D.r_cut * inv * u;
    float sm = 0.0f, sn = s1;                 // sin((n-1) th), sin(n th)
    for (int n = 0; n < D.n_basis; ++n) {
        Bcol[n * bstride] = pref * sn;
        float nx = 2.0f * c1 * sn - sm;
        sm = sn;
        sn = nx;
    }
}

// G matrices of one path for one edge.
// Floats per edge of the Y and dE/dY tiles (also ConvDesc::ys).
template <int LMAX>
constexpr int y_stride() { return LMAX >= 3 ? 16 : 9; }

// Only the couplings a kernel of degree LMAX can meet are compiled in.
template <int LMAX>
__device__ __forceinline__ void path_G(int kind, const float* Y, float* g) {
#define SN_G(a, b, c) case coupling_kind(a, b, c): CG<a, b, c>::G(Y + (b) * (b), g); break;
    if constexpr (LMAX <= 2) {
        switch (kind) {
            SN_FOR_EACH_COUPLING_L2(SN_G)
            default: break;
        }
    } else {
        switch (kind) {
            SN_FOR_EACH_COUPLING(SN_G)
            default: break;
        }
    }
#undef SN_G
}

// 4-byte asynchronous global -> shared copy (no register staging).
__device__ __forceinline__ void cp_async4(float* s, const float* g) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async16(float4* s, const float4* g) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Compile-time loop and the compile-time path list of one input irrep.
template <typename F, int... Is>
__device__ __forceinline__ void static_for_impl(F& f, std::integer_sequence<int, Is...>) {
    (f(std::integral_constant<int, Is>{}), ...);
}

template <int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

template <int L1, int LMAX, int KIND>
struct BlockPaths {
    static constexpr PathList list = path_list(L1, LMAX, KIND);
    static constexpr int begin = path_begin(L1, LMAX, KIND);
};

// ---- BF16 tensor-core variants of phases D and F (mma.sync m16n8k16, FP32 accumulate)
// The per-edge weight tile holds BF16 values in the BF16 forward kernel and
// FP32 values otherwise (the adjoint keeps dE/dw in FP32 beside w).
template <bool BF>
struct WTile {
    using T = float;
};
template <>
struct WTile<true> {
    using T = __nv_bfloat16;
};
__device__ __forceinline__ float wload(const float* p) { return *p; }
__device__ __forceinline__ float wload(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ void wstore(float* p, float v) { *p = v; }
__device__ __forceinline__ void wstore(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// The four floats of two packed BF16 pairs (a = (x, y), b = (z, w)).
__device__ __forceinline__ float4 unpack_bf16x4(uint32_t a, uint32_t b) {
    return make_float4(__uint_as_float(a << 16), __uint_as_float(a & 0xffff0000u), __uint_as_float(b << 16),
                       __uint_as_float(b & 0xffff0000u));
}

// Activations enter the tensor cores as one BF16 value (round to nearest).  W3
// is one BF16 value too; the hidden-layer weights W2 are a hi + lo BF16 pair
// (two MMAs), which keeps the virial error of the BF16 path near that of its
// forces (a single BF16 W2 raised it about fivefold).

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// The reduction order inside one MMA k step is free, so the BF16 products
// below permute k identically in the A and B fragments: lane (g, tq) owns the
// 32-bit words [tq * 2 KSN, (tq + 1) * 2 KSN) of every B row, which makes its B
// operand two contiguous 16-byte loads; k step ks then uses words
// w0 = tq * 2 KSN + 2 ks (first half of the fragment) and w0 + 1 (second half).

// Phase D (BF16): w[e][c] = sum_k H2[k][e] W3[k][c]; B operand W3T [W][H] (bf16).
// Each warp loads the B fragments of four n tiles at once.
template <int H, bool BFT>
__device__ __forceinline__ void chunk_w_gemm_bf16(const ConvDesc& D, const ConvSmem& L, float* smem,
                                                  const __nv_bfloat16* __restrict__ W3T) {
    constexpr int KSN = H / 16;                // k steps (4 or 2)
    constexpr int NV = KSN / 2;                // 16-byte loads per lane and n tile
    constexpr int BATCH = 4;
    static_assert(EC == 16, "one m tile of edges");
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, g = lane >> 2, tq = lane & 3;
    const float* s_H2 = smem + L.H2;
    uint32_t af[KSN][4];
#pragma unroll
    for (int ks = 0; ks < KSN; ++ks) {
        const int k0 = 2 * (tq * 2 * KSN + 2 * ks), k1 = k0 + 2;
        af[ks][0] = pack_bf16(s_H2[hk<H>(k0, g)], s_H2[hk<H>(k0 + 1, g)]);
        af[ks][1] = pack_bf16(s_H2[hk<H>(k0, g + 8)], s_H2[hk<H>(k0 + 1, g + 8)]);
        af[ks][2] = pack_bf16(s_H2[hk<H>(k1, g)], s_H2[hk<H>(k1 + 1, g)]);
        af[ks][3] = pack_bf16(s_H2[hk<H>(k1, g + 8)], s_H2[hk<H>(k1 + 1, g + 8)]);
    }
    const int ntiles = D.W / 8;
    for (int nb = warp; nb < ntiles; nb += BATCH * CONV_WARPS) {
        uint4 bv[BATCH][NV];
#pragma unroll
        for (int j = 0; j < BATCH; ++j) {
            const int nt = nb + j * CONV_WARPS;
            if (nt < ntiles) {
                const uint4* row = reinterpret_cast<const uint4*>(W3T + (size_t)(nt * 8 + g) * H);
#pragma unroll
                for (int v = 0; v < NV; ++v) bv[j][v] = __ldg(row + tq * NV + v);
            }
        }
#pragma unroll
        for (int j = 0; j < BATCH; ++j) {
            const int nt = nb + j * CONV_WARPS;
            if (nt >= ntiles) break;
            const uint32_t* bw = reinterpret_cast<const uint32_t*>(bv[j]);
            float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int ks = 0; ks < KSN; ++ks) {
                const uint32_t b[2] = {bw[2 * ks], bw[2 * ks + 1]};
                mma_bf16(c, af[ks], b);
            }
            const int col = nt * 8 + 2 * tq;
            if constexpr (BFT) {         // BF16 tile [EC][WpadB]
                __nv_bfloat16* s_w = reinterpret_cast<__nv_bfloat16*>(smem + L.w);
                *reinterpret_cast<__nv_bfloat162*>(s_w + g * D.WpadB + col) = __floats2bfloat162_rn(c[0], c[1]);
                *reinterpret_cast<__nv_bfloat162*>(s_w + (g + 8) * D.WpadB + col) =
                    __floats2bfloat162_rn(c[2], c[3]);
            } else {                     // FP32 tile [EC][Wpad]
                float* s_w = smem + L.w;
                *reinterpret_cast<float2*>(s_w + g * D.Wpad + col) = make_float2(c[0], c[1]);
                *reinterpret_cast<float2*>(s_w + (g + 8) * D.Wpad + col) = make_float2(c[2], c[3]);
            }
        }
    }
    __syncthreads();
}

// Phase F (BF16): gH2[k][e] = sum_c gw[e][c] W3[k][c]; B operand W3 [H][W] (bf16).
// K (the W columns, in blocks of 32) is split between four groups of two warps;
// within a group each warp owns H/16 n tiles of 8 hidden units for the group's
// whole K range, so every output has one writer per group.  Group 0 writes
// dE/dH2; groups 1-3 write partials into the dE/dw tile once every warp is done
// reading it (the BF16 adjoint's tile holds at least three [H][EC] partials),
// and the partials are added in group order, so the result does not depend on
// the warps' timing.
// SPLIT: dE/dw enters as a hi + lo BF16 pair (two MMAs per n tile), which keeps
// about 16 bits of it (the pair kernel's dE/dw is the sum of two directions).
template <int H, bool SPLIT = false>
__device__ __forceinline__ void chunk_gw_gemm_bf16(const ConvDesc& D, const ConvSmem& L, float* smem,
                                                   const __nv_bfloat16* __restrict__ W3h) {
    constexpr int G = 4, WPG = CONV_WARPS / G;
    constexpr int NTW = (H / 8) / WPG;         // n tiles per warp (4 or 2)
    static_assert(EC == 16, "one m tile of edges");
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, g = lane >> 2, tq = lane & 3;
    const int grp = warp / WPG, wq = warp % WPG;
    float* s_w = smem + L.w;                   // dE/dw, [EC][Wpad]
    float* s_gH = smem + L.gH;                 // [H][EC]
    const int W = D.W, nkb = W / 32;
    const int kb0 = nkb * grp / G, kb1 = nkb * (grp + 1) / G;
    __syncthreads();                           // every warp's dE/dw of phase E is in s_w
    float c[NTW][4];
#pragma unroll
    for (int j = 0; j < NTW; ++j) c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.f;
    for (int kb = kb0; kb < kb1; ++kb) {
        uint4 bv[NTW];
#pragma unroll
        for (int j = 0; j < NTW; ++j)
            bv[j] = __ldg(reinterpret_cast<const uint4*>(W3h + (size_t)((wq * NTW + j) * 8 + g) * W + kb * 32) + tq);
        // k step ks covers words kb*16 + 4 tq + 2 ks (+1): columns 32 kb + 8 tq + 4 ks .. + 3
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            const int c0 = kb * 32 + 8 * tq + 4 * ks;
            const float4 r0 = *reinterpret_cast<const float4*>(s_w + g * D.Wpad + c0);
            const float4 r1 = *reinterpret_cast<const float4*>(s_w + (g + 8) * D.Wpad + c0);
            const uint32_t a[4] = {pack_bf16(r0.x, r0.y), pack_bf16(r1.x, r1.y), pack_bf16(r0.z, r0.w),
                                   pack_bf16(r1.z, r1.w)};
            uint32_t al[4];
            if constexpr (SPLIT) {                 // the remainders x - bf16(x)
                const float4 h0 = unpack_bf16x4(a[0], a[2]), h1 = unpack_bf16x4(a[1], a[3]);
                al[0] = pack_bf16(r0.x - h0.x, r0.y - h0.y);
                al[1] = pack_bf16(r1.x - h1.x, r1.y - h1.y);
                al[2] = pack_bf16(r0.z - h0.z, r0.w - h0.w);
                al[3] = pack_bf16(r1.z - h1.z, r1.w - h1.w);
            }
#pragma unroll
            for (int j = 0; j < NTW; ++j) {
                const uint32_t* bw = reinterpret_cast<const uint32_t*>(&bv[j]);
                const uint32_t b[2] = {bw[2 * ks], bw[2 * ks + 1]};
                mma_bf16(c[j], a, b);
                if constexpr (SPLIT) mma_bf16(c[j], al, b);
            }
        }
    }
    __syncthreads();                           // the partials overwrite s_w
    float* out = grp == 0 ? s_gH : s_w + (grp - 1) * H * EC;
#pragma unroll
    for (int j = 0; j < NTW; ++j) {
        const int k = (wq * NTW + j) * 8 + 2 * tq;
        out[hk<H>(k, g)] = c[j][0];
        out[hk<H>(k + 1, g)] = c[j][1];
        out[hk<H>(k, g + 8)] = c[j][2];
        out[hk<H>(k + 1, g + 8)] = c[j][3];
    }
    __syncthreads();
    for (int i = t; i < H * EC; i += CONV_THREADS)
        s_gH[i] = ((s_gH[i] + s_w[i]) + s_w[H * EC + i]) + s_w[2 * H * EC + i];
    __syncthreads();
}

// Hidden layer of the radial MLP on tensor cores (BF16 path):
//   out[k_out][e] = sum_k in[k][e] B[k][k_out], B given N-major ([k_out][k]) as a
//   hi + lo BF16 pair, the input as one BF16 value; two MMAs per k step (in*hi, in*lo).
// The 16 edges of the chunk are one m tile; warps take n tiles of 8 outputs.
template <int H>
struct HiddenB {                                   // B fragments of one n tile, hi and lo
    uint4 hi[H / 32], lo[H / 32];
};

template <int H>
__device__ __forceinline__ void hidden_load(const __nv_bfloat16* __restrict__ Bn, int nt, HiddenB<H>& b) {
    constexpr int NV = H / 32;
    const int lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
    const uint4* hi = reinterpret_cast<const uint4*>(Bn + (size_t)(nt * 8 + g) * H) + tq * NV;
    const uint4* lo = reinterpret_cast<const uint4*>(Bn + (size_t)H * H + (size_t)(nt * 8 + g) * H) + tq * NV;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        b.hi[v] = __ldg(hi + v);
        b.lo[v] = __ldg(lo + v);
    }
}

// SPLIT: the input also enters as a hi + lo BF16 pair (in_lo * W2_hi added).
template <int H, bool SPLIT = false>
__device__ __forceinline__ void hidden_mma(const float* __restrict__ s_in, const HiddenB<H>& bf, float (&c)[4]) {
    constexpr int KSN = H / 16;
    const int lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
    c[0] = c[1] = c[2] = c[3] = 0.f;
    const uint32_t* wh = reinterpret_cast<const uint32_t*>(bf.hi);
    const uint32_t* wl = reinterpret_cast<const uint32_t*>(bf.lo);
#pragma unroll
    for (int ks = 0; ks < KSN; ++ks) {
        const int k0 = 2 * (tq * 2 * KSN + 2 * ks), k1 = k0 + 2;
        const uint32_t a[4] = {pack_bf16(s_in[hk<H>(k0, g)], s_in[hk<H>(k0 + 1, g)]),
                               pack_bf16(s_in[hk<H>(k0, g + 8)], s_in[hk<H>(k0 + 1, g + 8)]),
                               pack_bf16(s_in[hk<H>(k1, g)], s_in[hk<H>(k1 + 1, g)]),
                               pack_bf16(s_in[hk<H>(k1, g + 8)], s_in[hk<H>(k1 + 1, g + 8)])};
        const uint32_t b[2] = {wh[2 * ks], wh[2 * ks + 1]};
        const uint32_t b2[2] = {wl[2 * ks], wl[2 * ks + 1]};
        mma_bf16(c, a, b);
        mma_bf16(c, a, b2);
        if constexpr (SPLIT) {
            const float4 h0 = unpack_bf16x4(a[0], a[2]), h1 = unpack_bf16x4(a[1], a[3]);
            const uint32_t al[4] = {pack_bf16(s_in[hk<H>(k0, g)] - h0.x, s_in[hk<H>(k0 + 1, g)] - h0.y),
                                    pack_bf16(s_in[hk<H>(k0, g + 8)] - h1.x, s_in[hk<H>(k0 + 1, g + 8)] - h1.y),
                                    pack_bf16(s_in[hk<H>(k1, g)] - h0.z, s_in[hk<H>(k1 + 1, g)] - h0.w),
                                    pack_bf16(s_in[hk<H>(k1, g + 8)] - h1.z, s_in[hk<H>(k1 + 1, g + 8)] - h1.w)};
            mma_bf16(c, al, b);
        }
    }
}

// Phases A-C shared by both kernels.  Leaves s_src/s_dst/Y/B/A1/A2/H2/G filled.
// Edge data of one chunk, fetched one chunk ahead by threads 0..EC-1.
struct EdgePrefetch {
    int src = 0, dst = -1, first = 0;           // first: index of the receiver's first edge
    float4 geom = make_float4(0.f, 0.f, 0.f, 1.f);
    __device__ __forceinline__ void fetch(int c0, int E1, const int* __restrict__ dsts,
                                          const int* __restrict__ srcs, const float4* __restrict__ geoms,
                                          const int* __restrict__ row_ptr) {
        const int ge = c0 + (int)threadIdx.x;
        if ((int)threadIdx.x < EC && ge < E1) {
            src = srcs[ge];
            dst = dsts[ge];
            geom = geoms[ge];
            first = __ldg(row_ptr + dst);
        }
    }
};

// Radial MLP input layer into shared memory (once per CTA; the first chunk's
// barrier publishes it).
template <int H>
__device__ __forceinline__ void load_W1(const ConvDesc& D, const ConvSmem& L, float* smem,
                                        const float* __restrict__ W1) {
    for (int i = threadIdx.x; i < D.n_basis * H; i += CONV_THREADS) smem[L.W1 + i] = W1[i];
}

template <int H, bool BF, int LMAX>
__device__ __forceinline__ void chunk_prologue(const ConvDesc& D, const ConvSmem& L, float* smem,
                                               int c0, int ne, const EdgePrefetch& pf,
                                               const float* __restrict__ W2,
                                               const __nv_bfloat16* __restrict__ W2T_h) {
    const int t = threadIdx.x, warp = t >> 5;
    int* s_src = reinterpret_cast<int*>(smem + L.src);
    int* s_dst = reinterpret_cast<int*>(smem + L.dst);
    float* s_Y = smem + L.Y;
    float* s_B = smem + L.B;       // [NB][EC]
    if (t < EC) {
        if (t < ne) {
            s_src[t] = pf.src;
            s_dst[t] = pf.dst;
            reinterpret_cast<int*>(smem + L.first)[t] = pf.first >= c0;   // receiver starts here
            reinterpret_cast<float4*>(smem + L.geo)[t] = pf.geom;
            edge_features<LMAX>(D, pf.geom, s_Y + t * y_stride<LMAX>(), s_B + t, EC);
        } else {
            s_src[t] = 0;
            s_dst[t] = -1;
            reinterpret_cast<float4*>(smem + L.geo)[t] = make_float4(0.f, 0.f, 0.f, 1.f);
            for (int i = 0; i < y_stride<LMAX>(); ++i) s_Y[t * y_stride<LMAX>() + i] = 0.0f;
            for (int n = 0; n < D.n_basis; ++n) s_B[n * EC + t] = 0.0f;
        }
    }
    __syncthreads();
    // B: A1 = B @ W1 (layout [H][EC]); H1 = silu(A1) lives in the staging area until
    // phase D.  Thread (j, edge group): hidden unit j for EPT consecutive edges.
    float* s_A1 = smem + L.A1;
    float* s_A2 = smem + L.A2;
    float* s_H2 = smem + L.H2;
    float* s_H1 = smem + L.stage;
    {
        constexpr int EPT = EC * H / CONV_THREADS;
        static_assert(EPT == 4 || EPT == 2, "edges per thread of the input layer");
        static_assert(H / 8 <= CONV_WARPS, "one hidden n tile per warp");
        const int j = t % H, e0 = (t / H) * EPT;
        float a[EPT];
#pragma unroll
        for (int q = 0; q < EPT; ++q) a[q] = 0.0f;
        for (int n = 0; n < D.n_basis; ++n) {
            const float wv = smem[L.W1 + n * H + j];
            const float* bn = s_B + n * EC + e0;
#pragma unroll
            for (int q = 0; q < EPT; ++q) a[q] = fmaf(bn[q], wv, a[q]);
        }
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            const int o = hk<H>(j, e0 + q);
            s_A1[o] = a[q];
            s_H1[o] = siluf_(a[q]);
        }
    }
    // C: G matrices (independent of B)
    float* s_G = smem + L.G;
    for (int i = t; i < EC * D.n_paths; i += CONV_THREADS) {
        const int e = i % EC, p = i / EC;
        path_G<LMAX>(D.paths[p].kind, s_Y + e * y_stride<LMAX>(), s_G + e * D.nG + D.paths[p].g_off);
    }
    __syncthreads();
    if constexpr (BF) {          // A2 = H1 @ W2 on tensor cores, H2 = silu(A2)
        const int lane = t & 31, g = lane >> 2, tq = lane & 3;
        if (warp < H / 8) {
            const int nt = warp;
            float c[4];
            HiddenB<H> hb;
            hidden_load<H>(W2T_h, nt, hb);
            hidden_mma<H>(s_H1, hb, c);
            const int j = nt * 8 + 2 * tq;
            const int o[4] = {hk<H>(j, g), hk<H>(j + 1, g), hk<H>(j, g + 8), hk<H>(j + 1, g + 8)};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                s_A2[o[q]] = c[q];
                s_H2[o[q]] = siluf_(c[q]);
            }
        }
    } else {
        // A2 = H1 @ W2, H2 = silu(A2): each thread computes 4 hidden units of one edge
        for (int idx = t; idx < (H / 4) * EC; idx += CONV_THREADS) {
            const int jq = idx / EC, e = idx % EC;
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll 8
            for (int k = 0; k < H; ++k) {
                const float4 b = __ldg(reinterpret_cast<const float4*>(W2 + k * H) + jq);
                const float a = s_H1[hk<H>(k, e)];
                a0 = fmaf(a, b.x, a0);
                a1 = fmaf(a, b.y, a1);
                a2 = fmaf(a, b.z, a2);
                a3 = fmaf(a, b.w, a3);
            }
            const float av[4] = {a0, a1, a2, a3};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int o = hk<H>(4 * jq + q, e);
                s_A2[o] = av[q];
                s_H2[o] = siluf_(av[q]);
            }
        }
    }
    __syncthreads();
}

// Phase D (FP32): w[e][c] = sum_k H2[k][e] W3[k][c] for all W columns.
template <int H>
__device__ __forceinline__ void chunk_w_gemm_f32(const ConvDesc& D, const ConvSmem& L, float* smem,
                                                 const float* __restrict__ W3) {
    constexpr int NEG = EC / 4;                 // groups of 4 edges
    constexpr int NCG = CONV_THREADS / NEG;     // column-quad threads per edge group
    constexpr int NQ = DCOLS / (4 * NCG);       // column quads per thread and pass
    const int t = threadIdx.x;
    const int eg = t / NCG, cg = t % NCG;
    const float* s_H2 = smem + L.H2;
    float4* st4 = reinterpret_cast<float4*>(smem + L.stage);   // [KS][DCOLS/4]
    float* s_w = smem + L.w;
    const int W = D.W;
    for (int cb = 0; cb < W; cb += DCOLS) {
        float acc[4][NQ][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < NQ; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;
        for (int k0 = 0; k0 < H; k0 += KS) {
            __syncthreads();
            for (int i = t; i < KS * (DCOLS / 4); i += CONV_THREADS) {
                const int kk = i / (DCOLS / 4), q = i % (DCOLS / 4);
                const int col = cb + 4 * q;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (col < W) v = __ldg(reinterpret_cast<const float4*>(W3 + (size_t)(k0 + kk) * W + col));
                st4[i] = v;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < KS; ++kk) {
                const float4 a = *reinterpret_cast<const float4*>(s_H2 + hk<H>(k0 + kk, 4 * eg));
                const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
                for (int j = 0; j < NQ; ++j) {
                    const float4 b = st4[kk * (DCOLS / 4) + cg + NCG * j];
                    const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int q = 0; q < 4; ++q) acc[i][j][q] = fmaf(av[i], bv[q], acc[i][j][q]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < NQ; ++j) {
            const int col = cb + 4 * (cg + NCG * j);
            if (col < W) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    *reinterpret_cast<float4*>(s_w + (4 * eg + i) * D.Wpad + col) =
                        make_float4(acc[i][j][0], acc[i][j][1], acc[i][j][2], acc[i][j][3]);
            }
        }
    }
    __syncthreads();
}

// Receiver range of this CTA, balanced by edges.  The edge count is taken from
// row_ptr[n_atoms] (the host may not know it: asynchronous neighbour builds).
__device__ __forceinline__ void cta_range(int n_atoms, int /*n_edges*/, const int* __restrict__ row_ptr,
                                          int* s_range) {
    if (threadIdx.x == 0) {
        const int n_edges = row_ptr[n_atoms];
        const int nb = gridDim.x, b = blockIdx.x;
        auto lb = [&](long long key) {
            int lo = 0, hi = n_atoms;      // first v in [0, n_atoms] with row_ptr[v] >= key
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if ((long long)row_ptr[mid] < key) lo = mid + 1; else hi = mid;
            }
            return lo;
        };
        const long long elo = (long long)n_edges * b / nb;
        const long long ehi = (long long)n_edges * (b + 1) / nb;
        const int v0 = (b == 0) ? 0 : lb(elo);
        const int v1 = (b == nb - 1) ? n_atoms : lb(ehi);
        s_range[0] = v0;
        s_range[1] = v1;
    }
    __syncthreads();
}

// G matrix of one path into registers with 16-byte shared-memory loads
// (every path's G starts on a 16-byte boundary).
template <int NG>
__device__ __forceinline__ void load_G(const float* __restrict__ src, float* G) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int i = 0; i < (NG + 3) / 4; ++i) {
        const float4 v = s4[i];
        G[4 * i] = v.x;
        G[4 * i + 1] = v.y;
        G[4 * i + 2] = v.z;
        G[4 * i + 3] = v.w;
    }
}

template <int H>
__device__ __forceinline__ void chunk_gw_gemm_f32(const ConvDesc& D, const ConvSmem& L, float* smem,
                                                  const float* __restrict__ W3T) {
    constexpr int KQ = H / 4;                 // k quads
    constexpr int EGN = 128 / KQ;             // edge groups per half
    constexpr int EPT = EC / EGN;             // edges per thread
    const int t = threadIdx.x;
    const int half = t >> 7, tp = t & 127;
    const int kq = tp % KQ, eg = tp / KQ;
    const float* s_w = smem + L.w;
    float* stage = smem + L.stage;            // [2][CS][H]
    float acc[EPT][4];
#pragma unroll
    for (int i = 0; i < EPT; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] = 0.0f;
    const int W = D.W;
    for (int cb = 0; cb < W; cb += 2 * CS) {
        __syncthreads();
        for (int i = t; i < 2 * CS * (H / 4); i += CONV_THREADS) {
            const int hh = i / (CS * (H / 4));
            const int r = i % (CS * (H / 4));
            const int cc = r / (H / 4), k4 = r % (H / 4);
            const int c = cb + hh * CS + cc;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (c < W) v = __ldg(reinterpret_cast<const float4*>(W3T + (size_t)c * H) + k4);
            reinterpret_cast<float4*>(stage)[i] = v;
        }
        __syncthreads();
        const int cbase = cb + half * CS;
        const int cn = min(CS, W - cbase);
        const float* sh = stage + half * CS * H;
        for (int cc = 0; cc < cn; ++cc) {
            const float4 b = *reinterpret_cast<const float4*>(sh + cc * H + 4 * kq);
#pragma unroll
            for (int i = 0; i < EPT; ++i) {
                const float a = s_w[(eg * EPT + i) * D.Wpad + cbase + cc];
                acc[i][0] = fmaf(a, b.x, acc[i][0]);
                acc[i][1] = fmaf(a, b.y, acc[i][1]);
                acc[i][2] = fmaf(a, b.z, acc[i][2]);
                acc[i][3] = fmaf(a, b.w, acc[i][3]);
            }
        }
    }
    __syncthreads();
    float* red = stage;                       // [EC][H]
    if (half == 1) {
#pragma unroll
        for (int i = 0; i < EPT; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) red[(eg * EPT + i) * H + 4 * kq + q] = acc[i][q];
    }
    __syncthreads();
    float* s_gH = smem + L.gH;                // [H][EC]
    if (half == 0) {
#pragma unroll
        for (int i = 0; i < EPT; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int e = eg * EPT + i, k = 4 * kq + q;
                s_gH[hk<H>(k, e)] = acc[i][q] + red[e * H + k];
            }
    }
    __syncthreads();
}


static inline size_t smem_bytes(const ConvDesc& D, int H, bool bwd, bool bf) {
    return (size_t)conv_smem_layout(D.Wpad, D.WpadB, H, D.nG, D.ys, bwd, bf).total * sizeof(float);
}

static inline int conv_grid(int64_t n_atoms, int ctas_per_sm) {
    int dev = 0;
    cudaGetDevice(&dev);
    int g = ctas_per_sm * num_sms(dev);
    if (n_atoms < g) g = (int)(n_atoms > 0 ? n_atoms : 1);
    return g;
}

// Opt a kernel into `need` bytes of dynamic shared memory (never lowering a
// limit granted before in this process).
static inline sevennet_status conv_set_smem(const void* fn, size_t need, size_t* granted) {
    int dev = 0, optin = 0;
    SN_CUDA(cudaGetDevice(&dev));
    SN_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    need = need > *granted ? need : *granted;
    cudaFuncAttributes a{};
    SN_CUDA(cudaFuncGetAttributes(&a, fn));
    SN_CHECK(need + a.sharedSizeBytes <= (size_t)optin, SEVENNET_EINVAL,
             "convolution needs %zu bytes of shared memory, the device allows %d", need, optin);
    SN_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need));
    *granted = need;
    return SEVENNET_OK;
}

}  // namespace sn
