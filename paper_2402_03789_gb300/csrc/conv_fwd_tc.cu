// Forward tensor-product convolution of one interaction block on the tensor
// cores (BF16 path): Eq. 3 with the uvu product of Figure 2b.
//
// For path p = (l1, l2, l3), channel u and receiver v,
//   m_v[p][m3, u] = sum_{e into v} sum_{m1} (w_e[p, u] x_src(e)[l1][m1, u]) G_e^p[m1, m3],
//   G_e^p[m1, m3] = sum_{m2} C_p[m1, m2, m3] Y_l2(d_e)[m2].
// The inner sum over (e, m1) is a matrix product: for 16 channels (M), the m3
// of the path (N <= 8) and K = 16 slots of (edge, m1) pairs, mma.m16n8k16
// takes A[u][(e, m1)] = w_e[p, u] x_e[u, m1] and B[(e, m1)][m3] = G_e^p[m1, m3]
// in BF16 and accumulates in FP32.  The slots of one K group hold edges of one
// receiver (16 edges for l1 = 0, 4 for l1 = 1, 2 for l1 = 2), so the MMA
// accumulator carries the segmented sum over a receiver's edges; where a K
// group spans two receivers the MMA runs once per receiver with the other
// slots of A zeroed.  The accumulator is written when the receiver changes.
//
// Per 16-edge chunk: edge features (FP32), the x rows of the chunk's senders
// copied to shared memory by bulk copies (cp.async.bulk, completed on an
// mbarrier) while the radial MLP runs, the B
// fragments of every path built from Y, the hidden MLP layer and w^T = W3^T H2^T
// on mma.sync (w kept in BF16 as a [W][edge] tile), then the work units.
#include "conv_common.cuh"

namespace sn {

constexpr int TC_WS = 24;       // BF16 values between two columns of the [W][edge] weight tile (48 bytes: conflict-free lane patterns)

struct TcSmem {
    int w, xs, bf, stage, H2, Y, B, src, dst, first, W1, total;
};

__host__ __device__ inline TcSmem tc_smem_layout(const ConvDesc& D, int H) {
    TcSmem s;
    int o = 0;
    s.w = o;     o += rup4((D.W * TC_WS) / 2);
    s.xs = o;    o += D.xs_total;
    s.bf = o;    o += D.nBF;
    s.stage = o; o += (H * EC > MAX_NB * EC ? H * EC : MAX_NB * EC);
    s.H2 = o;    o += H * EC;
    s.Y = o;     o += EC * D.ys;
    s.B = o;     o += MAX_NB * EC;
    s.src = o;   o += EC;
    s.dst = o;   o += EC;
    s.first = o; o += EC;
    s.W1 = o;    o += MAX_NB * H;
    s.total = o;
    return s;
}

template <int L1, int LMAX, int KIND>
struct TcSets {
    static constexpr PathSets sets = tc_path_sets(L1, LMAX, KIND);
};

// ---- bulk copies (the TMA engine's linear mode) completed on an mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(a), "r"(bytes) : "memory");
}

// global -> shared, `bytes` a multiple of 16 and both addresses 16-byte aligned
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 ::"r"(d), "l"(src), "r"(bytes), "r"(b) : "memory");
}

// Wait for phase `parity` of the barrier to complete, for at most about `limit`
// clock cycles; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long long limit) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    const long long t0 = clock64();
    while (true) {
        unsigned done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) return false;
    }
}

constexpr long long TC_WAIT_LIMIT = 4000000000LL;   // about two seconds at 2 GHz

__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 v) { return *reinterpret_cast<uint32_t*>(&v); }
__device__ __forceinline__ __nv_bfloat162 bits_bf2(uint32_t v) { return *reinterpret_cast<__nv_bfloat162*>(&v); }
__device__ __forceinline__ uint32_t hmul2_bits(uint32_t a, uint32_t b) {
    return bf2_bits(__hmul2(bits_bf2(a), bits_bf2(b)));
}

// B fragments of one path for one edge: G[m1][m3] (FP32, from the sparse CG
// code) rounded to BF16 and stored where lane (g = m3, tq) of K group e / EG
// finds it.  Slot k of a K group: tq = (k & 7) / 2, register k / 8, half k & 1.
template <int L1, int L2, int L3>
__device__ __forceinline__ void tc_path_frag(const float* Y, int e, __nv_bfloat16* bf) {
    constexpr int N1 = 2 * L1 + 1, N3 = 2 * L3 + 1, EG = tc_eg(N1);
    float G[N1 * N3];
    CG<L1, L2, L3>::G(Y + L2 * L2, G);
    const int kg = e / EG, ej = e % EG;
    __nv_bfloat16* base = bf + kg * 128;
#pragma unroll
    for (int m1 = 0; m1 < N1; ++m1) {
        int tq, k;
        if constexpr (N1 == 1) { k = ej; tq = (k & 7) >> 1; }
        else if constexpr (N1 == 3) { tq = ej; k = 2 * tq + (m1 == 2 ? 8 : m1); }
        else { tq = 2 * ej + (m1 >> 2); const int q = m1 & 3; k = 2 * tq + 8 * (q >> 1) + (q & 1); }
        const int r = k >> 3, h = k & 1;
#pragma unroll
        for (int m3 = 0; m3 < N3; ++m3)
            base[(m3 * 4 + tq) * 4 + r * 2 + h] = __float2bfloat16_rn(G[m1 * N3 + m3]);
    }
}

template <int LMAX>
__device__ __forceinline__ void tc_frag_dispatch(int kind, const float* Y, int e, __nv_bfloat16* bf) {
#define SN_TCF(a, b, c) case coupling_kind(a, b, c): tc_path_frag<a, b, c>(Y, e, bf); break;
    switch (kind) {
        SN_FOR_EACH_COUPLING_L2(SN_TCF)
        default: break;
    }
#undef SN_TCF
}

// Phase D on tensor cores, transposed: w^T[c][e] = sum_k W3^T[c][k] H2[k][e],
// A = W3^T rows (the N-major BF16 copy of W3), B = H2 from the swizzled
// activation tile, stored as BF16 pairs of consecutive edges into [W][TC_WS].
// The k order inside an MMA is permuted identically in A and B so that each
// lane's A operand is one contiguous slice of its row.
template <int H>
__device__ __forceinline__ void tc_w_gemm(const ConvDesc& D, const TcSmem& L, float* smem,
                                          const __nv_bfloat16* __restrict__ W3T) {
    constexpr int KSN = H / 16, NV = KSN / 2;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, g = lane >> 2, tq = lane & 3;
    const float* s_H2 = smem + L.H2;
    uint32_t bh[2][KSN][2];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int ks = 0; ks < KSN; ++ks) {
            const int e = nt * 8 + g, k0 = 2 * (tq * 2 * KSN + 2 * ks);
            bh[nt][ks][0] = pack_bf16(s_H2[hk<H>(k0, e)], s_H2[hk<H>(k0 + 1, e)]);
            bh[nt][ks][1] = pack_bf16(s_H2[hk<H>(k0 + 2, e)], s_H2[hk<H>(k0 + 3, e)]);
        }
    uint32_t* s_w = reinterpret_cast<uint32_t*>(smem + L.w);      // word (c * TC_WS + e) / 2
    const int mtiles = D.W / 16;
    uint4 an[2][NV];                      // the next m tile's A operand, in flight during this tile's MMAs
    auto load_a = [&](int mt) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const uint4* row = reinterpret_cast<const uint4*>(W3T + (size_t)(mt * 16 + g + 8 * r) * H);
#pragma unroll
            for (int v = 0; v < NV; ++v) an[r][v] = __ldg(row + tq * NV + v);
        }
    };
    if (warp < mtiles) load_a(warp);
    for (int mt = warp; mt < mtiles; mt += CONV_WARPS) {
        uint4 av[2][NV];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int v = 0; v < NV; ++v) av[r][v] = an[r][v];
        if (mt + CONV_WARPS < mtiles) load_a(mt + CONV_WARPS);
        const uint32_t* a0w = reinterpret_cast<const uint32_t*>(av[0]);
        const uint32_t* a1w = reinterpret_cast<const uint32_t*>(av[1]);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int ks = 0; ks < KSN; ++ks) {
                const uint32_t a[4] = {a0w[2 * ks], a1w[2 * ks], a0w[2 * ks + 1], a1w[2 * ks + 1]};
                mma_bf16(c, a, bh[nt][ks]);
            }
            const int e = nt * 8 + 2 * tq;
            s_w[((mt * 16 + g) * TC_WS + e) >> 1] = pack_bf16(c[0], c[1]);
            s_w[((mt * 16 + g + 8) * TC_WS + e) >> 1] = pack_bf16(c[2], c[3]);
        }
    }
}

// One work unit: the paths [I0, I1) of input irrep L1 (set J) for channels
// u0 .. u0 + 15, over the chunk's edges.  Lane (g, tq) holds rows u0 + g and
// u0 + g + 8 of A and of the accumulators (columns m3 = 2 tq, 2 tq + 1).
template <int L1, int LMAX, int KIND, int J>
__device__ __forceinline__ void tc_unit(const ConvDesc& D, const TcSmem& L, const float* smem, int u0, int ne,
                                        unsigned segs, float* __restrict__ m) {
    using BP = BlockPaths<L1, LMAX, KIND>;
    constexpr int I0 = TcSets<L1, LMAX, KIND>::sets.b[J];
    constexpr int I1 = TcSets<L1, LMAX, KIND>::sets.b[J + 1];
    constexpr int NP = I1 - I0;
    constexpr int N1 = 2 * L1 + 1, EG = tc_eg(N1);
    const int lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
    const int* s_dst = reinterpret_cast<const int*>(smem + L.dst);
    const int* s_first = reinterpret_cast<const int*>(smem + L.first);
    const float* xs = smem + L.xs + D.xs_off[L1];
    const int xst = D.xs_stride[L1], mul = D.mul_in[L1], m_dim = D.m_dim;
    const __nv_bfloat16* wt = reinterpret_cast<const __nv_bfloat16*>(smem + L.w);
    const uint2* bfr = reinterpret_cast<const uint2*>(smem + L.bf);
    float acc[NP][4];
    // accumulator element (i, q) <-> path I0 + i, m3 = 2 tq + (q & 1), channel u0 + g + 8 (q >> 1)
    auto visit = [&](int v, auto&& f) {
        static_for<NP>([&](auto Ic) {
            constexpr int i = decltype(Ic)::value;
            constexpr int N3 = 2 * BP::list.l3[I0 + i] + 1;
            const PathDesc& P = D.paths[BP::begin + I0 + i];
            float* base = m + (size_t)v * m_dim + P.m_off + P.m_ch0 + u0 + g;
            if (2 * tq < N3) { f(base + 2 * tq * P.m_mul, acc[i][0]); f(base + 2 * tq * P.m_mul + 8, acc[i][2]); }
            if (2 * tq + 1 < N3) {
                f(base + (2 * tq + 1) * P.m_mul, acc[i][1]);
                f(base + (2 * tq + 1) * P.m_mul + 8, acc[i][3]);
            }
        });
    };
    auto zero = [&]() {
#pragma unroll
        for (int i = 0; i < NP; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.0f;
    };
    zero();
    int cur = s_dst[0];
    if (!s_first[0]) visit(cur, [](float* p, float& a) { a = *p; });   // carried over from the previous chunk
    for (int e_lo = 0; e_lo < ne; e_lo += EG) {
        const int ke = min(e_lo + EG, ne);
        // this lane's x values (FP32 from the staged rows) packed to BF16 pairs, rows u0 + g (+ 8)
        uint32_t xp[2][2];
        int el[4];
        if constexpr (N1 == 1) {
            el[0] = 2 * tq; el[1] = 2 * tq + 1; el[2] = 2 * tq + 8; el[3] = 2 * tq + 9;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const float* xr = xs + u0 + g + 8 * r;
                xp[r][0] = pack_bf16(xr[el[0] * xst], xr[el[1] * xst]);
                xp[r][1] = pack_bf16(xr[el[2] * xst], xr[el[3] * xst]);
            }
        } else {
            const int e = e_lo + (N1 == 3 ? tq : (tq >> 1));
            el[0] = e;
            const int mb = N1 == 3 ? 0 : 4 * (tq & 1);
            const int q3 = N1 == 3 ? 2 : mb + 2;      // m1 of the second register's first half
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const float* xr = xs + e * xst + u0 + g + 8 * r;
                float v0, v1, v2, v3;
                if constexpr (N1 == 3) {
                    v0 = xr[0]; v1 = xr[mul]; v2 = xr[2 * mul]; v3 = 0.0f;
                } else {
                    v0 = mb < N1 ? xr[mb * mul] : 0.0f;
                    v1 = mb + 1 < N1 ? xr[(mb + 1) * mul] : 0.0f;
                    v2 = q3 < N1 ? xr[q3 * mul] : 0.0f;
                    v3 = q3 + 1 < N1 ? xr[(q3 + 1) * mul] : 0.0f;
                }
                xp[r][0] = pack_bf16(v0, v1);
                xp[r][1] = pack_bf16(v2, v3);
            }
        }
        // per path: B fragments and the weights w_e[p, u] of this lane's edges
        uint2 bq[NP];
        uint32_t wr[NP][2][2];
        static_for<NP>([&](auto Ic) {
            constexpr int i = decltype(Ic)::value;
            const PathDesc& P = D.paths[BP::begin + I0 + i];
            bq[i] = bfr[(P.b_off >> 1) + (e_lo / EG) * 32 + lane];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const __nv_bfloat16* wc = wt + (P.col0 + u0 + g + 8 * r) * TC_WS;
                if constexpr (N1 == 1) {
                    wr[i][r][0] = *reinterpret_cast<const uint32_t*>(wc + 2 * tq);
                    wr[i][r][1] = *reinterpret_cast<const uint32_t*>(wc + 2 * tq + 8);
                } else {
                    const uint32_t b = bf2_bits(__bfloat162bfloat162(wc[el[0]]));
                    wr[i][r][0] = b;
                    wr[i][r][1] = b;
                }
            }
        });
        // receiver runs inside this K group
        int rs = e_lo;
        while (rs < ke) {
            const unsigned later = segs & ~((2u << rs) - 1u);
            const int re = later ? min(__ffs(later) - 1, ke) : ke;
            const int v = s_dst[rs];
            if (v != cur) {
                visit(cur, [](float* p, float& a) { *p = a; });
                cur = v;
                zero();
            }
            uint32_t xa[2][2];
            if constexpr (N1 == 1) {
                const uint32_t k0 = (el[0] >= rs && el[0] < re ? 0xFFFFu : 0u) |
                                    (el[1] >= rs && el[1] < re ? 0xFFFF0000u : 0u);
                const uint32_t k1 = (el[2] >= rs && el[2] < re ? 0xFFFFu : 0u) |
                                    (el[3] >= rs && el[3] < re ? 0xFFFF0000u : 0u);
#pragma unroll
                for (int r = 0; r < 2; ++r) { xa[r][0] = xp[r][0] & k0; xa[r][1] = xp[r][1] & k1; }
            } else {
                const bool in = el[0] >= rs && el[0] < re;
#pragma unroll
                for (int r = 0; r < 2; ++r) { xa[r][0] = in ? xp[r][0] : 0u; xa[r][1] = in ? xp[r][1] : 0u; }
            }
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                const uint32_t a[4] = {hmul2_bits(xa[0][0], wr[i][0][0]), hmul2_bits(xa[1][0], wr[i][1][0]),
                                       hmul2_bits(xa[0][1], wr[i][0][1]), hmul2_bits(xa[1][1], wr[i][1][1])};
                const uint32_t b[2] = {bq[i].x, bq[i].y};
                mma_bf16(acc[i], a, b);
            }
            rs = re;
        }
    }
    if (ne > 0) visit(cur, [](float* p, float& a) { *p = a; });
}

template <int H, int LMAX, int KIND>
__device__ __forceinline__ void tc_chunk(const ConvDesc& D, const TcSmem& L, const float* smem, int ne,
                                         unsigned segs, float* __restrict__ m) {
    const int warp = threadIdx.x >> 5;
    for (int s = 0; s < D.n_slots_tc[warp]; ++s) {
        const int code = D.slot_tc[warp][s];
        const int l1 = code >> 12, set = (code >> 8) & 15, u0 = (code & 255) * 16;
        static_for<LMAX + 1>([&](auto Lc) {
            constexpr int L1 = decltype(Lc)::value;
            static_for<TC_MAX_SETS>([&](auto Jc) {
                constexpr int J = decltype(Jc)::value;
                if constexpr (J < TcSets<L1, LMAX, KIND>::sets.n) {
                    if (l1 == L1 && set == J) tc_unit<L1, LMAX, KIND, J>(D, L, smem, u0, ne, segs, m);
                }
            });
        });
    }
}

template <int H, int LMAX>
__global__ void __launch_bounds__(CONV_THREADS, 2)
conv_fwd_tc_kernel(const ConvDesc D, const float* __restrict__ W1, const __nv_bfloat16* __restrict__ W3T_h,
                   const __nv_bfloat16* __restrict__ W2T_h, int n_atoms, int n_edges,
                   const int* __restrict__ row_ptr, const int* __restrict__ dst, const int* __restrict__ src,
                   const float4* __restrict__ geom, const float* __restrict__ x, float* __restrict__ m,
                   int* flags) {
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    const TcSmem L = tc_smem_layout(D, H);
    __shared__ int s_range[2];
    __shared__ __align__(8) uint64_t s_bar;           // completion of the chunk's x-row copies
    if (threadIdx.x == 0) mbar_init(&s_bar, 1);
    cta_range(n_atoms, n_edges, row_ptr, s_range);
    const int v0 = s_range[0], v1 = s_range[1];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int v = v0 + warp; v < v1; v += CONV_WARPS) {       // receivers without edges get zero messages
        if (row_ptr[v] == row_ptr[v + 1]) {
            for (int i = lane; i < D.m_dim; i += 32) m[(size_t)v * D.m_dim + i] = 0.0f;
        }
    }
    const int E0 = row_ptr[v0], E1 = row_ptr[v1];
    int* s_src = reinterpret_cast<int*>(smem + L.src);
    int* s_dst = reinterpret_cast<int*>(smem + L.dst);
    int* s_first = reinterpret_cast<int*>(smem + L.first);
    float* s_Y = smem + L.Y;
    float* s_B = smem + L.B;
    float* s_H1 = smem + L.stage;
    float* s_H2 = smem + L.H2;
    __nv_bfloat16* s_bf = reinterpret_cast<__nv_bfloat16*>(smem + L.bf);
    // B-fragment slots that no path writes (m3 beyond the path, padding slots) stay zero
    for (int i = t; i < D.nBF; i += CONV_THREADS) smem[L.bf + i] = 0.0f;
    for (int i = t; i < D.n_basis * H; i += CONV_THREADS) smem[L.W1 + i] = W1[i];
    // bytes of the x rows of one edge (each irrep's block is copied to its own region)
    unsigned row_bytes = 0;
#pragma unroll
    for (int l = 0; l < NL; ++l) row_bytes += (unsigned)((2 * l + 1) * D.mul_in[l]) * 4u;
    unsigned parity = 0;
    EdgePrefetch pf;
    pf.fetch(E0, E1, dst, src, geom, row_ptr);
    for (int c0 = E0; c0 < E1; c0 += EC) {
        const int ne = min(EC, E1 - c0);
        __syncthreads();
        if (t == 0) mbar_expect_tx(&s_bar, row_bytes * (unsigned)ne);   // this chunk's x-row bytes
        if (t < EC) {
            if (t < ne) {
                s_src[t] = pf.src;
                s_dst[t] = pf.dst;
                s_first[t] = pf.first >= c0;
                edge_features<LMAX>(D, pf.geom, s_Y + t * D.ys, s_B + t, EC);
            } else {
                s_src[t] = 0;
                s_dst[t] = -1;
                s_first[t] = 1;
                for (int i = 0; i < D.ys; ++i) s_Y[t * D.ys + i] = 0.0f;
                for (int n = 0; n < D.n_basis; ++n) s_B[n * EC + t] = 0.0f;
            }
        }
        __syncthreads();
        // x rows of the chunk's senders into shared memory by bulk copies (one per
        // edge and irrep), in flight during the MLP; the previous chunk's reads of
        // these regions ended at the barrier above
        if (lane < NL && D.mul_in[lane]) {           // lane l of warp w copies irrep l of edges w, w + 8
            const int l = lane;
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            for (int e = warp; e < ne; e += CONV_WARPS)
                bulk_copy(smem + L.xs + D.xs_off[l] + e * D.xs_stride[l], x + (size_t)s_src[e] * D.x_dim + D.x_off[l],
                          (unsigned)((2 * l + 1) * D.mul_in[l]) * 4u, &s_bar);
        }
        // radial MLP input layer: H1 = silu(B @ W1), thread (j, edge group)
        {
            constexpr int EPT = EC * H / CONV_THREADS;
            const int j = t % H, e0 = (t / H) * EPT;
            float a[EPT];
#pragma unroll
            for (int q = 0; q < EPT; ++q) a[q] = 0.0f;
            for (int n = 0; n < D.n_basis; ++n) {
                const float wv = smem[L.W1 + n * H + j];
#pragma unroll
                for (int q = 0; q < EPT; ++q) a[q] = fmaf(s_B[n * EC + e0 + q], wv, a[q]);
            }
#pragma unroll
            for (int q = 0; q < EPT; ++q) s_H1[hk<H>(j, e0 + q)] = siluf_(a[q]);
        }
        // B fragments of every path
        for (int i = t; i < EC * D.n_paths; i += CONV_THREADS) {
            const int e = i % EC, p = i / EC;
            tc_frag_dispatch<LMAX>(D.paths[p].kind, s_Y + e * D.ys, e, s_bf + 2 * D.paths[p].b_off);
        }
        __syncthreads();
        if (warp < H / 8) {       // hidden layer on tensor cores: H2 = silu(H1 @ W2)
            const int g = lane >> 2, tq = lane & 3, nt = warp;
            float c[4];
            HiddenB<H> hb;
            hidden_load<H>(W2T_h, nt, hb);
            hidden_mma<H>(s_H1, hb, c);
            const int j = nt * 8 + 2 * tq;
            s_H2[hk<H>(j, g)] = siluf_(c[0]);
            s_H2[hk<H>(j + 1, g)] = siluf_(c[1]);
            s_H2[hk<H>(j, g + 8)] = siluf_(c[2]);
            s_H2[hk<H>(j + 1, g + 8)] = siluf_(c[3]);
        }
        pf.fetch(c0 + EC, E1, dst, src, geom, row_ptr);
        __syncthreads();
        tc_w_gemm<H>(D, L, smem, W3T_h);
        // the x rows have landed (bounded wait: a copy that never completes is
        // reported in flags[FLAG_COPY_TIMEOUT] and the CTA's messages are left NaN)
        const bool ok = mbar_wait(&s_bar, parity, TC_WAIT_LIMIT);
        parity ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (t == 0 && flags) atomicOr(flags + FLAG_COPY_TIMEOUT, 1);
            mbar_wait(&s_bar, parity ^ 1u, TC_WAIT_LIMIT);          // once more for the copies in flight
            for (int v = v0 + warp; v < v1; v += CONV_WARPS)
                for (int i = lane; i < D.m_dim; i += 32) m[(size_t)v * D.m_dim + i] = __int_as_float(0x7fc00000);
            return;
        }
        // receiver boundaries of the chunk: bit e set where a receiver's run starts
        const unsigned segs = __ballot_sync(0xffffffffu, lane < ne && (lane == 0 || s_dst[lane] != s_dst[lane - 1]));
        switch (D.kind) {
            case 0: tc_chunk<H, LMAX, 0>(D, L, smem, ne, segs, m); break;
            case 1: tc_chunk<H, LMAX, 1>(D, L, smem, ne, segs, m); break;
            case 2: tc_chunk<H, LMAX, 2>(D, L, smem, ne, segs, m); break;
            default: tc_chunk<H, LMAX, 3>(D, L, smem, ne, segs, m); break;
        }
    }
}

size_t conv_tc_smem_bytes(const ConvDesc& D, int H) { return (size_t)tc_smem_layout(D, H).total * sizeof(float); }

sevennet_status conv_configure_fwd_tc(int H, size_t need) {
    static size_t granted[2] = {0, 0};
    if (H == 64) {
        SN_TRY(conv_set_smem((const void*)conv_fwd_tc_kernel<64, 1>, need, &granted[1]));
        SN_TRY(conv_set_smem((const void*)conv_fwd_tc_kernel<64, 2>, need, &granted[1]));
    } else if (H == 32) {
        SN_TRY(conv_set_smem((const void*)conv_fwd_tc_kernel<32, 1>, need, &granted[0]));
        SN_TRY(conv_set_smem((const void*)conv_fwd_tc_kernel<32, 2>, need, &granted[0]));
    }
    return SEVENNET_OK;
}

void launch_conv_fwd_tc(const LayerDev& Ld, int H, int64_t n_atoms, int64_t n_edges, const int* row_ptr,
                        const int* dst, const int* src, const float4* geom, const float* x, float* m,
                        int* flags, cudaStream_t st) {
    const int grid = conv_grid(n_atoms, 2);
    const size_t sm = conv_tc_smem_bytes(Ld.conv, H);
#define SN_LT(HH, LL) conv_fwd_tc_kernel<HH, LL><<<grid, CONV_THREADS, sm, st>>>(                     \
        Ld.conv, Ld.mlp0, Ld.mlp2h, Ld.mlp1Th, (int)n_atoms, (int)n_edges, row_ptr, dst, src, geom, x, m, flags)
    if (H == 64) { if (Ld.conv.lmax == 2) SN_LT(64, 2); else SN_LT(64, 1); }
    else { if (Ld.conv.lmax == 2) SN_LT(32, 2); else SN_LT(32, 1); }
#undef SN_LT
}

}  // namespace sn
