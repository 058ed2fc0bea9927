// Tensor-product convolution of one interaction block and its adjoint.
//
// Forward (paper Eq. 3, Figure 2b; SevenNet-0 details Sec. 5.1):
//   m_v[p][m3, u] = sum_{e into v} w_e[p, u] sum_{m1} x_src(e)[l1][m1, u] G_e^p[m1, m3]
//   G_e^p[m1, m3] = sum_{m2} C_p[m1, m2, m3] Y_l2(d_e)[m2],
//   w_e = MLP(Bessel(r_e) * envelope(r_e))  (the 1/avg_num_neigh factor is folded into
//   the last MLP weight matrix on the host).
// Adjoint (Eqs. 5-8): given g_m = dE/dm, each edge produces dE/dx_src (scattered
// to the sender with vector-free FP32 reductions), dE/dw_e -> back through the
// MLP to dE/dr_e, and dE/dY_e; together dE/dd_e, accumulated over blocks.
//
// One CTA owns a contiguous range of receivers (balanced by edge count) and
// walks its edges, sorted by receiver, in chunks of EC edges.  Per chunk:
//   A  geometry: r, unit vector, Y (l <= 2), Bessel basis x envelope  (FP32)
//   B  radial MLP hidden layers                                      (FFMA)
//   C  G matrices of every path for every edge of the chunk
//   D  w = H2 @ W3 for all W columns into shared memory              (FFMA)
//   E  forward: each warp owns 32-channel groups of paths and walks the edges,
//      keeping the running sum of the current receiver in registers and writing
//      it once when the receiver changes (segmented sum, no atomics);
//      adjoint: each warp owns edges and walks all paths of that edge.
#include "internal.h"
#include "cg_tables.cuh"

namespace sn {

constexpr int KS = 8;         // k-slice of the W3 staging in phase D
constexpr int DCOLS = 512;    // columns per pass of phase D
constexpr int CS = 32;        // column slice of phase F (adjoint W3 product)

struct ConvSmem {
    int w, stage, A1, A2, H2, gH, G, Y, B, gY, src, dst, total;
};

__host__ __device__ inline int rup4(int x) { return (x + 3) & ~3; }

__host__ __device__ inline ConvSmem conv_smem_layout(int Wpad, int H, int nG, bool bwd) {
    ConvSmem s;
    int o = 0;
    s.w = o;     o += EC * Wpad;
    s.stage = o; o += (KS * DCOLS > 2 * CS * 64 ? KS * DCOLS : 2 * CS * 64);
    s.A1 = o;    o += H * EC;
    s.A2 = o;    o += H * EC;
    s.H2 = o;    o += H * EC;
    s.gH = o;    o += bwd ? H * EC : 0;
    s.G = o;     o += rup4(EC * nG);
    s.Y = o;     o += EC * 9;
    s.B = o;     o += MAX_NB * EC;
    s.gY = o;    o += bwd ? EC * 9 : 0;
    s.src = o;   o += EC;
    s.dst = o;   o += EC;
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
__device__ __forceinline__ void path_G(int kind, const float* Y, float* g) {
    switch (kind) {
#define SN_G(a, b, c) case coupling_kind(a, b, c): CG<a, b, c>::G(Y + (b) * (b), g); break;
        SN_G(0, 0, 0) SN_G(0, 1, 1) SN_G(0, 2, 2)
        SN_G(1, 0, 1) SN_G(1, 1, 0) SN_G(1, 1, 1) SN_G(1, 1, 2) SN_G(1, 2, 1) SN_G(1, 2, 2)
        SN_G(2, 0, 2) SN_G(2, 1, 1) SN_G(2, 1, 2) SN_G(2, 2, 0) SN_G(2, 2, 1) SN_G(2, 2, 2)
#undef SN_G
        default: break;
    }
}

// ---- BF16 tensor-core variants of phases D and F (mma.sync m16n8k16, FP32 accumulate)
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// Activations enter the tensor cores as hi + lo BF16 pairs (two MMAs), weights as
// one BF16 value: the product keeps ~16 mantissa bits of the activation.
constexpr bool SPLIT_ACT = true;

__device__ __forceinline__ void split_bf16(float x, float y, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(x - hf.x, y - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Phase D (BF16): w[e][c] = sum_k H2[k][e] W3[k][c]; B operand W3T [W][H] (bf16).
template <int H>
__device__ __forceinline__ void chunk_w_gemm_bf16(const ConvDesc& D, const ConvSmem& L, float* smem,
                                                  const __nv_bfloat16* __restrict__ W3T) {
    constexpr int KSN = H / 16;
    constexpr int MT = EC / 16;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, g = lane >> 2, tq = lane & 3;
    const float* s_H2 = smem + L.H2;
    float* s_w = smem + L.w;
    uint32_t af[MT][KSN][4], al[MT][KSN][4];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int ks = 0; ks < KSN; ++ks) {
            const int k0 = ks * 16 + 2 * tq, e0 = mt * 16 + g;
            split_bf16(s_H2[k0 * EC + e0], s_H2[(k0 + 1) * EC + e0], af[mt][ks][0], al[mt][ks][0]);
            split_bf16(s_H2[k0 * EC + e0 + 8], s_H2[(k0 + 1) * EC + e0 + 8], af[mt][ks][1], al[mt][ks][1]);
            split_bf16(s_H2[(k0 + 8) * EC + e0], s_H2[(k0 + 9) * EC + e0], af[mt][ks][2], al[mt][ks][2]);
            split_bf16(s_H2[(k0 + 8) * EC + e0 + 8], s_H2[(k0 + 9) * EC + e0 + 8], af[mt][ks][3], al[mt][ks][3]);
        }
    const int ntiles = D.W / 8;
    uint32_t bn[KSN][2];
    auto loadb = [&](int nt, uint32_t (*b)[2]) {
        const uint32_t* row = reinterpret_cast<const uint32_t*>(W3T + (size_t)(nt * 8 + g) * H);
#pragma unroll
        for (int ks = 0; ks < KSN; ++ks) {
            b[ks][0] = __ldg(row + ks * 8 + tq);
            b[ks][1] = __ldg(row + ks * 8 + 4 + tq);
        }
    };
    if (warp < ntiles) loadb(warp, bn);
    for (int nt = warp; nt < ntiles; nt += CONV_WARPS) {
        uint32_t bc[KSN][2];
#pragma unroll
        for (int ks = 0; ks < KSN; ++ks) { bc[ks][0] = bn[ks][0]; bc[ks][1] = bn[ks][1]; }
        if (nt + CONV_WARPS < ntiles) loadb(nt + CONV_WARPS, bn);
        float c[MT][4];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) c[mt][0] = c[mt][1] = c[mt][2] = c[mt][3] = 0.f;
#pragma unroll
        for (int ks = 0; ks < KSN; ++ks)
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                mma_bf16(c[mt], af[mt][ks], bc[ks]);
                if constexpr (SPLIT_ACT) mma_bf16(c[mt], al[mt][ks], bc[ks]);
            }
        const int col = nt * 8 + 2 * tq;
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
            const int r = mt * 16 + g;
            *reinterpret_cast<float2*>(s_w + r * D.Wpad + col) = make_float2(c[mt][0], c[mt][1]);
            *reinterpret_cast<float2*>(s_w + (r + 8) * D.Wpad + col) = make_float2(c[mt][2], c[mt][3]);
        }
    }
    __syncthreads();
}

// Phase F (BF16): gH2[k][e] = sum_c gw[e][c] W3[k][c]; B operand W3 [H][W] (bf16).
// The K (column) range is split over the warps, so each dE/dw fragment is read
// and split once; partial sums meet in shared memory.
template <int H>
__device__ __forceinline__ void chunk_gw_gemm_bf16(const ConvDesc& D, const ConvSmem& L, float* smem,
                                                   const __nv_bfloat16* __restrict__ W3h) {
    constexpr int NT = H / 8;                  // n tiles of 8 hidden units
    static_assert(EC == 16, "one m tile of edges");
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, g = lane >> 2, tq = lane & 3;
    const float* s_w = smem + L.w;
    float* s_gH = smem + L.gH;                 // [H][EC]
    const int W = D.W;
    for (int i = t; i < H * EC; i += CONV_THREADS) s_gH[i] = 0.0f;
    __syncthreads();
    float c[NT][4];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.f;
    for (int ks = warp; ks < W / 16; ks += CONV_WARPS) {
        const int c0 = ks * 16 + 2 * tq;
        const float2 x0 = *reinterpret_cast<const float2*>(s_w + g * D.Wpad + c0);
        const float2 x1 = *reinterpret_cast<const float2*>(s_w + (g + 8) * D.Wpad + c0);
        const float2 x2 = *reinterpret_cast<const float2*>(s_w + g * D.Wpad + c0 + 8);
        const float2 x3 = *reinterpret_cast<const float2*>(s_w + (g + 8) * D.Wpad + c0 + 8);
        uint32_t a[4], al[4];
        split_bf16(x0.x, x0.y, a[0], al[0]);
        split_bf16(x1.x, x1.y, a[1], al[1]);
        split_bf16(x2.x, x2.y, a[2], al[2]);
        split_bf16(x3.x, x3.y, a[3], al[3]);
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const uint32_t* brow = reinterpret_cast<const uint32_t*>(W3h + (size_t)(nt * 8 + g) * W);
            const uint32_t b[2] = {__ldg(brow + (c0 >> 1)), __ldg(brow + ((c0 + 8) >> 1))};
            mma_bf16(c[nt], a, b);
            if constexpr (SPLIT_ACT) mma_bf16(c[nt], al, b);
        }
    }
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        const int k = nt * 8 + 2 * tq;
        atomicAdd(s_gH + k * EC + g, c[nt][0]);
        atomicAdd(s_gH + (k + 1) * EC + g, c[nt][1]);
        atomicAdd(s_gH + k * EC + g + 8, c[nt][2]);
        atomicAdd(s_gH + (k + 1) * EC + g + 8, c[nt][3]);
    }
    __syncthreads();
}

// Hidden layer of the radial MLP on tensor cores (BF16 path):
//   out[k_out][e] = sum_k in[k][e] B[k][k_out], B given N-major ([k_out][k]) as a
//   hi + lo BF16 pair; three MMAs per k step (hi*hi, lo*hi, hi*lo).
// The 16 edges of the chunk are one m tile; warps take n tiles of 8 outputs.
template <int H>
__device__ __forceinline__ void hidden_mma(const float* __restrict__ s_in, const __nv_bfloat16* __restrict__ Bn,
                                           float (&c)[4], int nt) {
    constexpr int KSN = H / 16;
    const int lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
    c[0] = c[1] = c[2] = c[3] = 0.f;
    const uint32_t* brow = reinterpret_cast<const uint32_t*>(Bn + (size_t)(nt * 8 + g) * H);
#pragma unroll
    for (int ks = 0; ks < KSN; ++ks) {
        const int k0 = ks * 16 + 2 * tq;
        uint32_t a[4], al[4];
        split_bf16(s_in[k0 * EC + g], s_in[(k0 + 1) * EC + g], a[0], al[0]);
        split_bf16(s_in[k0 * EC + g + 8], s_in[(k0 + 1) * EC + g + 8], a[1], al[1]);
        split_bf16(s_in[(k0 + 8) * EC + g], s_in[(k0 + 9) * EC + g], a[2], al[2]);
        split_bf16(s_in[(k0 + 8) * EC + g + 8], s_in[(k0 + 9) * EC + g + 8], a[3], al[3]);
        const uint32_t b[2] = {__ldg(brow + (k0 >> 1)), __ldg(brow + ((k0 + 8) >> 1))};
        const uint32_t bl[2] = {__ldg(brow + H * H / 2 + (k0 >> 1)), __ldg(brow + H * H / 2 + ((k0 + 8) >> 1))};
        mma_bf16(c, a, b);
        if constexpr (SPLIT_ACT) mma_bf16(c, al, b);
        mma_bf16(c, a, bl);
    }
}

// Phases A-C shared by both kernels.  Leaves s_src/s_dst/Y/B/A1/A2/H2/G filled.
template <int H, bool BF>
__device__ __forceinline__ void chunk_prologue(const ConvDesc& D, const ConvSmem& L, float* smem,
                                               int c0, int ne, const int* __restrict__ dst,
                                               const int* __restrict__ src,
                                               const float4* __restrict__ geom,
                                               const float* __restrict__ W1,
                                               const float* __restrict__ W2,
                                               const __nv_bfloat16* __restrict__ W2T_h) {
    const int t = threadIdx.x;
    int* s_src = reinterpret_cast<int*>(smem + L.src);
    int* s_dst = reinterpret_cast<int*>(smem + L.dst);
    float* s_Y = smem + L.Y;
    float* s_B = smem + L.B;       // [NB][EC]
    if (t < EC) {
        if (t < ne) {
            const int ge = c0 + t;
            s_src[t] = src[ge];
            s_dst[t] = dst[ge];
            edge_features(D, geom[ge], s_Y + t * 9, s_B + t, EC);
        } else {
            s_src[t] = 0;
            s_dst[t] = -1;
            for (int i = 0; i < 9; ++i) s_Y[t * 9 + i] = 0.0f;
            for (int n = 0; n < D.n_basis; ++n) s_B[n * EC + t] = 0.0f;
        }
    }
    __syncthreads();
    // B: A1 = B @ W1 (layout [H][EC]); H1 = silu(A1) lives in the staging area until phase D
    float* s_A1 = smem + L.A1;
    float* s_A2 = smem + L.A2;
    float* s_H2 = smem + L.H2;
    float* s_H1 = smem + L.stage;
    for (int i = t; i < H * EC; i += CONV_THREADS) {
        const int j = i / EC, e = i % EC;
        float a = 0.0f;
        for (int n = 0; n < D.n_basis; ++n) a = fmaf(s_B[n * EC + e], __ldg(W1 + n * H + j), a);
        s_A1[i] = a;
        s_H1[i] = siluf_(a);
    }
    // C: G matrices (independent of B)
    float* s_G = smem + L.G;
    for (int i = t; i < EC * D.n_paths; i += CONV_THREADS) {
        const int e = i % EC, p = i / EC;
        path_G(D.paths[p].kind, s_Y + e * 9, s_G + e * D.nG + D.paths[p].g_off);
    }
    __syncthreads();
    if constexpr (BF) {          // A2 = H1 @ W2 on tensor cores, H2 = silu(A2)
        const int warp = t >> 5, lane = t & 31, g = lane >> 2, tq = lane & 3;
        for (int nt = warp; nt < H / 8; nt += CONV_WARPS) {
            float c[4];
            hidden_mma<H>(s_H1, W2T_h, c, nt);
            const int j = nt * 8 + 2 * tq;
            const int o[4] = {j * EC + g, (j + 1) * EC + g, j * EC + g + 8, (j + 1) * EC + g + 8};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                s_A2[o[q]] = c[q];
                s_H2[o[q]] = siluf_(c[q]);
            }
        }
        __syncthreads();
        return;
    }
    // A2 = H1 @ W2, H2 = silu(A2): each thread computes 4 hidden units of one edge
    for (int idx = t; idx < (H / 4) * EC; idx += CONV_THREADS) {
        const int jq = idx / EC, e = idx % EC;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll 8
        for (int k = 0; k < H; ++k) {
            const float4 b = __ldg(reinterpret_cast<const float4*>(W2 + k * H) + jq);
            const float a = s_H1[k * EC + e];
            a0 = fmaf(a, b.x, a0);
            a1 = fmaf(a, b.y, a1);
            a2 = fmaf(a, b.z, a2);
            a3 = fmaf(a, b.w, a3);
        }
        const float av[4] = {a0, a1, a2, a3};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int o = (4 * jq + q) * EC + e;
            s_A2[o] = av[q];
            s_H2[o] = siluf_(av[q]);
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
                const float4 a = *reinterpret_cast<const float4*>(s_H2 + (k0 + kk) * EC + 4 * eg);
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

// Receiver range of this CTA, balanced by edges.
__device__ __forceinline__ void cta_range(int n_atoms, int n_edges, const int* __restrict__ row_ptr,
                                          int* s_range) {
    if (threadIdx.x == 0) {
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

// ------------------------------------------------------------- forward
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

template <int L1, int L2, int L3>
__device__ __forceinline__ void tp_fwd_group(const PathDesc& P, int u, int c0, int ne,
                                             const float* s_w, int Wpad, const float* s_G, int nG,
                                             const int* s_src, const int* s_dst,
                                             const int* __restrict__ row_ptr,
                                             const float* __restrict__ x, int x_dim,
                                             float* __restrict__ m, int m_dim) {
    constexpr int N1 = 2 * L1 + 1, N3 = 2 * L3 + 1;
    const int col = P.col0 + u;
    const float* xb = x + P.x_off + u;
    float* mb = m + P.m_off + P.m_ch0 + u;
    float acc[N3];
#pragma unroll
    for (int c = 0; c < N3; ++c) acc[c] = 0.0f;
    int cur = -1;
    auto flush = [&](int v) {
        float* mp = mb + (size_t)v * m_dim;
        if (__ldg(row_ptr + v) >= c0) {
#pragma unroll
            for (int c = 0; c < N3; ++c) mp[c * P.m_mul] = acc[c];
        } else {
#pragma unroll
            for (int c = 0; c < N3; ++c) mp[c * P.m_mul] += acc[c];
        }
    };
    constexpr int PF = 4;       // edges whose gathers are in flight together
    for (int e0 = 0; e0 < ne; e0 += PF) {
        float xv[PF][N1];
#pragma unroll
        for (int q = 0; q < PF; ++q) {
            const int e = min(e0 + q, ne - 1);
            const float* xr = xb + (size_t)s_src[e] * x_dim;
#pragma unroll
            for (int a = 0; a < N1; ++a) xv[q][a] = __ldg(xr + a * P.mul);
        }
#pragma unroll
        for (int q = 0; q < PF; ++q) {
            const int e = e0 + q;
            if (e >= ne) break;
            const int v = s_dst[e];
            if (v != cur) {
                if (cur >= 0) flush(cur);
                cur = v;
#pragma unroll
                for (int c = 0; c < N3; ++c) acc[c] = 0.0f;
            }
            const float wv = s_w[e * Wpad + col];
            float G[((N1 * N3 + 3) / 4) * 4];
            load_G<N1 * N3>(s_G + e * nG + P.g_off, G);
#pragma unroll
            for (int c = 0; c < N3; ++c) {
                float tt = 0.0f;
#pragma unroll
                for (int a = 0; a < N1; ++a) tt = fmaf(xv[q][a], G[a * N3 + c], tt);
                acc[c] = fmaf(wv, tt, acc[c]);
            }
        }
    }
    if (cur >= 0) flush(cur);
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
    for (int c0 = E0; c0 < E1; c0 += EC) {
        const int ne = min(EC, E1 - c0);
        __syncthreads();
        chunk_prologue<H, BF>(D, L, smem, c0, ne, dst, src, geom, W1, W2, W2T_h);
        if constexpr (BF) chunk_w_gemm_bf16<H>(D, L, smem, W3T_h);
        else chunk_w_gemm_f32<H>(D, L, smem, W3);
        for (int s = 0; s < D.n_slots[warp]; ++s) {
            const int g = D.slot_group[warp][s];
            const PathDesc& P = D.paths[g >> 8];
            const int u = (g & 255) * 32 + lane;
            switch (P.kind) {
#define SN_F(a, b, c) case coupling_kind(a, b, c):                                              \
                tp_fwd_group<a, b, c>(P, u, c0, ne, smem + L.w, D.Wpad, smem + L.G, D.nG, s_src, \
                                      s_dst, row_ptr, x, D.x_dim, m, D.m_dim); break;
                SN_F(0, 0, 0) SN_F(0, 1, 1) SN_F(0, 2, 2)
                SN_F(1, 0, 1) SN_F(1, 1, 0) SN_F(1, 1, 1) SN_F(1, 1, 2) SN_F(1, 2, 1) SN_F(1, 2, 2)
                SN_F(2, 0, 2) SN_F(2, 1, 1) SN_F(2, 1, 2) SN_F(2, 2, 0) SN_F(2, 2, 1) SN_F(2, 2, 2)
#undef SN_F
                default: break;
            }
        }
    }
}

// ------------------------------------------------------------- adjoint
template <int L1, int L2, int L3>
__device__ __forceinline__ void tp_bwd_path(const PathDesc& P, int u, int e, int v, const float* xv,
                                            float* gx, float* gY, float* s_w, int Wpad,
                                            const float* s_G, int nG,
                                            const float* __restrict__ gm, int m_dim) {
    constexpr int N1 = 2 * L1 + 1, N3 = 2 * L3 + 1;
    const int col = P.col0 + u;
    const float* gmr = gm + (size_t)v * m_dim + P.m_off + P.m_ch0 + u;
    float g[N3];
#pragma unroll
    for (int c = 0; c < N3; ++c) g[c] = __ldg(gmr + c * P.m_mul);
    const float wv = s_w[e * Wpad + col];
    float G[((N1 * N3 + 3) / 4) * 4];
    load_G<N1 * N3>(s_G + e * nG + P.g_off, G);
    float q[N1];
    float gw = 0.0f;
#pragma unroll
    for (int a = 0; a < N1; ++a) {
        float tt = 0.0f;
#pragma unroll
        for (int c = 0; c < N3; ++c) tt = fmaf(G[a * N3 + c], g[c], tt);
        q[a] = tt;
        gw = fmaf(xv[a], tt, gw);
        gx[a] = fmaf(wv, tt, gx[a]);
    }
    s_w[e * Wpad + col] = gw;        // dE/dw replaces w (same thread, same slot)
    float wx[N1];
#pragma unroll
    for (int a = 0; a < N1; ++a) wx[a] = wv * xv[a];
    CG<L1, L2, L3>::gY(wx, g, gY + L2 * L2);
}

template <int L1>
__device__ __forceinline__ void tp_bwd_l1(const ConvDesc& D, int lane, int e, int v, int sidx,
                                          float* gY, float* s_w, const float* s_G,
                                          const float* __restrict__ x,
                                          const float* __restrict__ gm, float* __restrict__ gxo) {
    constexpr int N1 = 2 * L1 + 1;
    const int mul = D.mul_in[L1];
    const float* xr = x + (size_t)sidx * D.x_dim + D.x_off[L1];
    float* gxr = gxo + (size_t)sidx * D.x_dim + D.x_off[L1];
    for (int ub = 0; ub < mul; ub += 32) {
        const int u = ub + lane;
        float xv[N1], gx[N1];
#pragma unroll
        for (int a = 0; a < N1; ++a) {
            xv[a] = __ldg(xr + a * mul + u);
            gx[a] = 0.0f;
        }
        for (int p = D.pbeg[L1]; p < D.pend[L1]; ++p) {
            const PathDesc& P = D.paths[p];
            switch (P.l2 * 3 + P.l3) {
#define SN_B(b, c)                                                                                  \
                case (b) * 3 + (c):                                                                 \
                    if constexpr (((L1 > b ? L1 - b : b - L1) <= c) && (c <= L1 + b) && c <= 2)     \
                        tp_bwd_path<L1, b, c>(P, u, e, v, xv, gx, gY, s_w, D.Wpad, s_G, D.nG, gm,   \
                                              D.m_dim);                                             \
                    break;
                SN_B(0, 0) SN_B(0, 1) SN_B(0, 2) SN_B(1, 0) SN_B(1, 1) SN_B(1, 2) SN_B(2, 0)
                SN_B(2, 1) SN_B(2, 2)
#undef SN_B
                default: break;
            }
        }
#pragma unroll
        for (int a = 0; a < N1; ++a) atomicAdd(gxr + a * mul + u, gx[a]);
    }
}

// Phase F (FP32): gH2[k][e] = sum_c gw[e][c] W3T[c][k], split over two thread halves.
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
                s_gH[k * EC + e] = acc[i][q] + red[e * H + k];
            }
    }
    __syncthreads();
}

template <int H, bool BF>
__global__ void __launch_bounds__(CONV_THREADS, 2)
conv_bwd_kernel(const ConvDesc D, const float* __restrict__ W1, const float* __restrict__ W2,
                const float* __restrict__ W2T, const float* __restrict__ W3, const float* __restrict__ W3T,
                const __nv_bfloat16* __restrict__ W3T_h, const __nv_bfloat16* __restrict__ W3_h,
                const __nv_bfloat16* __restrict__ W2T_h, const __nv_bfloat16* __restrict__ W2_h,
                int n_atoms,
                int n_edges, const int* __restrict__ row_ptr, const int* __restrict__ dst,
                const int* __restrict__ src, const float4* __restrict__ geom,
                const float* __restrict__ x, const float* __restrict__ gm,
                float* __restrict__ gx, float* __restrict__ gd) {
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    const ConvSmem L = conv_smem_layout(D.Wpad, H, D.nG, true);
    __shared__ int s_range[2];
    cta_range(n_atoms, n_edges, row_ptr, s_range);
    const int v0 = s_range[0], v1 = s_range[1];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int E0 = row_ptr[v0], E1 = row_ptr[v1];
    const int* s_src = reinterpret_cast<const int*>(smem + L.src);
    const int* s_dst = reinterpret_cast<const int*>(smem + L.dst);
    float* s_w = smem + L.w;
    float* s_gY = smem + L.gY;
    for (int c0 = E0; c0 < E1; c0 += EC) {
        const int ne = min(EC, E1 - c0);
        __syncthreads();
        chunk_prologue<H, BF>(D, L, smem, c0, ne, dst, src, geom, W1, W2, W2T_h);
        if constexpr (BF) chunk_w_gemm_bf16<H>(D, L, smem, W3T_h);
        else chunk_w_gemm_f32<H>(D, L, smem, W3);
        // E: per-edge adjoint of the tensor product
        for (int e = warp; e < ne; e += CONV_WARPS) {
            const int v = s_dst[e], sidx = s_src[e];
            float gY[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) gY[i] = 0.0f;
            if (D.mul_in[0]) tp_bwd_l1<0>(D, lane, e, v, sidx, gY, s_w, smem + L.G, x, gm, gx);
            if (D.mul_in[1]) tp_bwd_l1<1>(D, lane, e, v, sidx, gY, s_w, smem + L.G, x, gm, gx);
            if (D.mul_in[2]) tp_bwd_l1<2>(D, lane, e, v, sidx, gY, s_w, smem + L.G, x, gm, gx);
#pragma unroll
            for (int i = 0; i < 9; ++i) gY[i] = warp_sum(gY[i]);
            if (lane < 9) {
                float val = gY[0];
#pragma unroll
                for (int i = 1; i < 9; ++i) if (lane == i) val = gY[i];
                s_gY[e * 9 + lane] = val;
            }
        }
        // F: dE/dH2 = dE/dw @ W3^T
        if constexpr (BF) chunk_gw_gemm_bf16<H>(D, L, smem, W3_h);
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
            if (nt < H / 8) hidden_mma<H>(s_gH, W2_h, c, nt);
            __syncthreads();       // every read of A2 (the silu' above) is done
            if (nt < H / 8) {
                const int k = nt * 8 + 2 * tq;
                const int o[4] = {k * EC + g, (k + 1) * EC + g, k * EC + g + 8, (k + 1) * EC + g + 8};
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
                    const float a = s_gH[j * EC + e];
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
                    const int o = (4 * kq + q) * EC + e;
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
            for (int k = 0; k < H; ++k) a = fmaf(s_A2[k * EC + e], __ldg(W1 + n * H + k), a);
            s_gB[i] = a;
        }
        __syncthreads();
        // G: dE/dd = (dE/dr) u + (I - u u^T) dE/du / r
        if (t < ne) {
            const float4 g = geom[c0 + t];
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
            const float* gy = s_gY + t * 9;
            const float s3 = 1.7320508075688772f, s15 = 3.872983346207417f, s5 = 2.23606797749979f;
            float gux = s3 * gy[3], guy = s3 * gy[1], guz = s3 * gy[2];
            if (D.lmax >= 2) {
                gux += s15 * (uy * gy[4] + uz * gy[7] + ux * gy[8]);
                guy += s15 * (ux * gy[4] + uz * gy[5] - uy * gy[8]);
                guz += s15 * (uy * gy[5] + ux * gy[7]) + 3.0f * s5 * uz * gy[6];
            }
            const float dot = gux * ux + guy * uy + guz * uz;
            float* o = gd + (size_t)(c0 + t) * 3;
            o[0] += dEdr * ux + (gux - dot * ux) * inv;
            o[1] += dEdr * uy + (guy - dot * uy) * inv;
            o[2] += dEdr * uz + (guz - dot * uz) * inv;
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

// ------------------------------------------------------------- launchers
static size_t smem_bytes(const ConvDesc& D, int H, bool bwd) {
    return (size_t)conv_smem_layout(D.Wpad, H, D.nG, bwd).total * sizeof(float);
}

// Opt the convolution kernels into the shared memory the model's blocks need.
sevennet_status conv_configure(int H, const std::vector<LayerDev>& layers) {
    int dev = 0;
    SN_CUDA(cudaGetDevice(&dev));
    int optin = 0;
    SN_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    size_t need_f = 0, need_b = 0;
    for (const LayerDev& L : layers) {
        need_f = std::max(need_f, smem_bytes(L.conv, H, false));
        need_b = std::max(need_b, smem_bytes(L.conv, H, true));
    }
    // never lower a limit another model of the process relies on
    static size_t granted[2][2] = {{0, 0}, {0, 0}};
    const int hi = (H == 64) ? 1 : 0;
    need_f = std::max(need_f, granted[hi][0]);
    need_b = std::max(need_b, granted[hi][1]);
    granted[hi][0] = need_f;
    granted[hi][1] = need_b;
    auto set = [&](const void* fn, size_t need) -> sevennet_status {
        cudaFuncAttributes a{};
        SN_CUDA(cudaFuncGetAttributes(&a, fn));
        SN_CHECK(need + a.sharedSizeBytes <= (size_t)optin, SEVENNET_EINVAL,
                 "convolution needs %zu bytes of shared memory, the device allows %d", need, optin);
        SN_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need));
        return SEVENNET_OK;
    };
    if (H == 64) {
        SN_TRY(set((const void*)conv_fwd_kernel<64, false>, need_f));
        SN_TRY(set((const void*)conv_bwd_kernel<64, false>, need_b));
        SN_TRY(set((const void*)conv_fwd_kernel<64, true>, need_f));
        SN_TRY(set((const void*)conv_bwd_kernel<64, true>, need_b));
    } else if (H == 32) {
        SN_TRY(set((const void*)conv_fwd_kernel<32, false>, need_f));
        SN_TRY(set((const void*)conv_bwd_kernel<32, false>, need_b));
        SN_TRY(set((const void*)conv_fwd_kernel<32, true>, need_f));
        SN_TRY(set((const void*)conv_bwd_kernel<32, true>, need_b));
    } else {
        set_error("radial MLP hidden width must be 32 or 64");
        return SEVENNET_EINVAL;
    }
    return SEVENNET_OK;
}

size_t conv_smem_need(const ConvDesc& D, int H) { return smem_bytes(D, H, true); }

static int conv_grid(int64_t n_atoms) {
    int dev = 0;
    cudaGetDevice(&dev);
    int g = 2 * num_sms(dev);                 // two CTAs per SM
    if (n_atoms < g) g = (int)(n_atoms > 0 ? n_atoms : 1);
    return g;
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

void launch_conv_bwd(const LayerDev& L, int H, sevennet_precision prec, int64_t n_atoms,
                     int64_t n_edges, const int* row_ptr, const int* dst, const int* src,
                     const float4* geom, const float* x, const float* gm, float* gx,
                     float* gd, cudaStream_t st) {
    const int grid = conv_grid(n_atoms);
    const size_t sm = smem_bytes(L.conv, H, true);
    const bool bf = prec == SEVENNET_BF16;
#define SN_LB(HH, BB) conv_bwd_kernel<HH, BB><<<grid, CONV_THREADS, sm, st>>>(                     \
        L.conv, L.mlp0, L.mlp1, L.mlp1T, L.mlp2, L.mlp2T, L.mlp2h, L.mlp2Th, L.mlp1Th, L.mlp1h,       \
        (int)n_atoms,                                                                                 \
        (int)n_edges, row_ptr, dst, src, geom, x, gm, gx, gd)
    if (H == 64) { if (bf) SN_LB(64, true); else SN_LB(64, false); }
    else         { if (bf) SN_LB(32, true); else SN_LB(32, false); }
#undef SN_LB
}

}  // namespace sn
