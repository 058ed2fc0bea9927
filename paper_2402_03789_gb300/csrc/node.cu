// Node-level kernels of the interaction blocks and the readout.
//
//  * per-irrep linears (linear_1, self-connection, linear_2; Figure 2b and the
//    self-connection-as-linear of Sec. 5.1): out[v, m, :] = in[v, m, :] @ W,
//    W pre-scaled by 1/sqrt(fan_in); rows are (atom, m) pairs.
//  * gate (NequIP's equivariant nonlinearity, Sec. 3.2) and its adjoint.
//  * embedding h1 = W_emb[Z] and the atomwise readout (Eq. 1).
//  * forces F_v = sum_w (F_vw - F_wv) (Eq. 6) from the per-edge gradients
//    F_vw = dE/dd_vw accumulated over blocks (Eq. 5), and the atom virials
//    -sum_e F_e (x) d_e, both summed in FP64.
#include "internal.h"

namespace sn {

__device__ __forceinline__ float sigm(float x) { return 1.0f / (1.0f + expf(-x)); }
__device__ __forceinline__ float silu_(float x) { return x * sigm(x); }
__device__ __forceinline__ float dsilu_(float x) {
    float s = sigm(x);
    return s * (1.0f + x * (1.0f - s));
}

// ---------------------------------------------------------------- FP32 GEMM
// 64 x 64 output tile, 256 threads, 4 x 4 per thread, K slices of 16.
__global__ void __launch_bounds__(256)
gemm_f32_kernel(const GemmBatch batch) {
    const GemmProb& P = batch.p[blockIdx.z];
    const int64_t rows = P.n_atoms * P.R;
    const int64_t r0 = (int64_t)blockIdx.x * 64;
    const int n0 = blockIdx.y * 64;
    if (r0 >= rows || n0 >= P.N) return;
    __shared__ __align__(16) float sA[16][68];
    __shared__ __align__(16) float sB[16][64];
    const int t = threadIdx.x;
    const int tr = t / 16, tc = t % 16;
    float acc[4][4] = {};
    // A loader: row = t / 4 (0..63), k quad = t % 4
    const int lrow = t / 4, lkq = t % 4;
    const int64_t arow = r0 + lrow;
    const float* aptr = nullptr;
    if (arow < rows) {
        const int64_t v = arow / P.R;
        const int mm = (int)(arow % P.R);
        aptr = P.A + v * P.lda + P.a_off + (int64_t)mm * P.K;
    }
    const int bk = t / 16, bc = t % 16;
    for (int k0 = 0; k0 < P.K; k0 += 16) {
        float4 av = make_float4(0.f, 0.f, 0.f, 0.f);
        if (aptr) av = *reinterpret_cast<const float4*>(aptr + k0 + 4 * lkq);
        sA[4 * lkq + 0][lrow] = av.x;
        sA[4 * lkq + 1][lrow] = av.y;
        sA[4 * lkq + 2][lrow] = av.z;
        sA[4 * lkq + 3][lrow] = av.w;
        float4 bv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (n0 + 4 * bc < P.N)
            bv = __ldg(reinterpret_cast<const float4*>(P.B + (int64_t)(k0 + bk) * P.N + n0 + 4 * bc));
        *reinterpret_cast<float4*>(&sB[bk][4 * bc]) = bv;
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const float4 a = *reinterpret_cast<const float4*>(&sA[kk][4 * tr]);
            const float4 b = *reinterpret_cast<const float4*>(&sB[kk][4 * tc]);
            const float aa[4] = {a.x, a.y, a.z, a.w};
            const float bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(aa[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
    const int col = n0 + 4 * tc;
    if (col >= P.N) return;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t row = r0 + 4 * tr + i;
        if (row >= rows) break;
        const int64_t v = row / P.R;
        const int mm = (int)(row % P.R);
        float* cp = P.C + v * P.ldc + P.c_off + (int64_t)mm * P.N + col;
        float4 o = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
        if (P.accumulate) {
            const float4 c = *reinterpret_cast<const float4*>(cp);
            o.x += c.x; o.y += c.y; o.z += c.z; o.w += c.w;
        }
        *reinterpret_cast<float4*>(cp) = o;
    }
}

// ---------------------------------------------------------------- BF16 GEMM
// Tensor cores (mma.sync m16n8k16, BF16 operands, FP32 accumulate).  A is read
// as FP32 and rounded to BF16 in the fragment; B is the BF16 [N][K] copy.
// Activations and weights both enter as hi + lo BF16 pairs; three MMAs
// (hi*hi, lo*hi, hi*lo) keep about 16 mantissa bits of each operand.
constexpr bool GEMM_SPLIT_ACT = true;

__device__ __forceinline__ void split_bf16_n(float x, float y, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(x - hf.x, y - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

__device__ __forceinline__ void mma_bf16_n(float* c, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// 128 x 64 output tile, 8 warps as 4 (rows) x 2 (cols), each warp 32 rows x 32
// cols (2 m tiles x 4 n tiles); for N <= 32 the warps stack 8 x 1 over 256 x 32.
// K runs in blocks of 32 under one k permutation of both operands (the
// reduction order inside an MMA is free): lane tq owns
// k = kb + 8 tq + [0, 8), k step ks takes kb + 8 tq + 4 ks + [0, 4).  Its A
// values are then one float4 per row and k step, and its B words (hi and lo)
// one 16-byte load per n row and k block.  K and N are multiples of 32.
__global__ void __launch_bounds__(256)
gemm_bf16_kernel(const GemmBatch batch) {
    const GemmProb& P = batch.p[blockIdx.z];
    const int64_t rows = P.n_atoms * P.R;
    // N <= 32: the 8 warps stack as 8 x 1 over a 256 x 32 tile (the grid's extra
    // row blocks exit); otherwise 4 x 2 over 128 x 64
    const bool narrow = P.N <= 32;
    const int64_t r0 = (int64_t)blockIdx.x * (narrow ? 256 : 128);
    const int n0 = blockIdx.y * 64;
    if (r0 >= rows || n0 >= P.N) return;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, g = lane >> 2, tq = lane & 3;
    const int wr = narrow ? warp : (warp & 3), wc = narrow ? 0 : (warp >> 2);
    const int nbase = n0 + wc * 32;
    if (nbase >= P.N) return;
    auto rowptr = [&](int64_t r) -> const float* {
        if (r >= rows) return nullptr;
        const int64_t v = r / P.R;
        const int mm = (int)(r % P.R);
        return P.A + v * P.lda + P.a_off + (int64_t)mm * P.K;
    };
    const float* pr[2][2];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h) pr[mt][h] = rowptr(r0 + wr * 32 + mt * 16 + h * 8 + g);
    float c[2][4][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int j = 0; j < 4; ++j) c[mt][j][0] = c[mt][j][1] = c[mt][j][2] = c[mt][j][3] = 0.0f;
    const int64_t lo_off = (int64_t)P.K * P.N;          // bf16 elements
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int kb = 0; kb < P.K; kb += 32) {
        uint4 bh[4], bl[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const __nv_bfloat16* br = P.Bh + (int64_t)(nbase + j * 8 + g) * P.K + kb + 8 * tq;
            bh[j] = __ldg(reinterpret_cast<const uint4*>(br));
            bl[j] = __ldg(reinterpret_cast<const uint4*>(br + lo_off));
        }
        float4 av[2][2][2];                                // [m tile][row half][k step]
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int ks = 0; ks < 2; ++ks)
                    av[mt][h][ks] = pr[mt][h] ? *reinterpret_cast<const float4*>(pr[mt][h] + kb + 8 * tq + 4 * ks) : z4;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                uint32_t a[4], al[4];
                split_bf16_n(av[mt][0][ks].x, av[mt][0][ks].y, a[0], al[0]);
                split_bf16_n(av[mt][1][ks].x, av[mt][1][ks].y, a[1], al[1]);
                split_bf16_n(av[mt][0][ks].z, av[mt][0][ks].w, a[2], al[2]);
                split_bf16_n(av[mt][1][ks].z, av[mt][1][ks].w, a[3], al[3]);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t* wh = reinterpret_cast<const uint32_t*>(&bh[j]);
                    const uint32_t* wl = reinterpret_cast<const uint32_t*>(&bl[j]);
                    const uint32_t b[2] = {wh[2 * ks], wh[2 * ks + 1]};
                    const uint32_t b2[2] = {wl[2 * ks], wl[2 * ks + 1]};
                    mma_bf16_n(c[mt][j], a, b);
                    if (GEMM_SPLIT_ACT) mma_bf16_n(c[mt][j], al, b);
                    mma_bf16_n(c[mt][j], a, b2);
                }
            }
        }
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t r = r0 + wr * 32 + mt * 16 + h * 8 + g;
            if (r >= rows) continue;
            const int64_t v = r / P.R;
            const int mm = (int)(r % P.R);
            float* cp = P.C + v * P.ldc + P.c_off + (int64_t)mm * P.N;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int col = nbase + j * 8 + 2 * tq;
                float2 o = make_float2(c[mt][j][2 * h], c[mt][j][2 * h + 1]);
                if (P.accumulate) {
                    const float2 q = *reinterpret_cast<const float2*>(cp + col);
                    o.x += q.x;
                    o.y += q.y;
                }
                *reinterpret_cast<float2*>(cp + col) = o;
            }
        }
}

void launch_gemm(const GemmBatch& b, sevennet_precision prec, cudaStream_t st) {
    if (b.n == 0) return;
    int64_t max_rows = 0;
    int max_n = 0;
    for (int i = 0; i < b.n; ++i) {
        max_rows = std::max<int64_t>(max_rows, b.p[i].n_atoms * b.p[i].R);
        max_n = std::max(max_n, b.p[i].N);
    }
    if (max_rows == 0) return;
    if (prec == SEVENNET_BF16) {
        const dim3 grid((unsigned)((max_rows + 127) / 128), (unsigned)((max_n + 63) / 64), (unsigned)b.n);
        gemm_bf16_kernel<<<grid, 256, 0, st>>>(b);
    } else {
        const dim3 grid((unsigned)((max_rows + 63) / 64), (unsigned)((max_n + 63) / 64), (unsigned)b.n);
        gemm_f32_kernel<<<grid, 256, 0, st>>>(b);
    }
}

// ---------------------------------------------------------------- embedding
__device__ __forceinline__ int clamp_species(int s, int ns) { return s < 0 ? 0 : (s >= ns ? ns - 1 : s); }

// Out-of-range species are clamped here (no out-of-bounds read) and reported
// as an error by the host after the evaluation.
__global__ void embed_kernel(const float* __restrict__ table, const int* __restrict__ species,
                             int64_t n, int mul0, int n_species, float* __restrict__ h) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * mul0) return;
    const int64_t v = i / mul0;
    const int u = (int)(i % mul0);
    h[i] = table[(int64_t)clamp_species(species[v], n_species) * mul0 + u];
}

void launch_embed(const float* table, const int* species, int64_t n, int mul0, int n_species, float* h,
                  cudaStream_t st) {
    const int64_t tot = n * mul0;
    if (tot == 0) return;
    embed_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(table, species, n, mul0, n_species, h);
}

// ---------------------------------------------------------------- gate
struct GateDims {
    int mul0, ng, lmax, y_dim, h_dim;
    int mul[NL], y_off[NL], h_off[NL], goff[NL];
    int last;
};

// Entry l (1..3) of a per-irrep array of the kernel parameter, by selects: a
// dynamic index into a by-value parameter array would copy it to local memory.
__device__ __forceinline__ int irrep_sel(const int (&a)[NL], int l) {
    return l == 1 ? a[1] : (l == 2 ? a[2] : a[3]);
}

static GateDims gate_dims(const LayerDev& L, int mul0, const int* mul, int lmax) {
    GateDims g{};
    g.mul0 = mul0;
    g.lmax = lmax;
    g.y_dim = L.y_dim;
    g.h_dim = L.h_out_dim;
    g.last = L.last ? 1 : 0;
    int go = 0;
    for (int l = 0; l < NL; ++l) {
        g.mul[l] = (l <= lmax) ? mul[l] : 0;
        g.y_off[l] = L.y_off[l];
        g.h_off[l] = L.out_off[l];
        if (l >= 1 && l <= lmax) { g.goff[l] = go; go += mul[l]; }
    }
    g.ng = go;
    return g;
}

// The gate kernels walk atoms (grid-stride) with the CTA's threads over one
// atom's row, so no element index is divided by a row length.
static inline unsigned gate_grid(int64_t n) {
    int dev = 0;
    cudaGetDevice(&dev);
    const int64_t g = (int64_t)8 * num_sms(dev);
    return (unsigned)(n < g ? n : g);
}

__global__ void gate_fwd_kernel(const GateDims G, int64_t n, const float* __restrict__ y,
                                float* __restrict__ h) {
    for (int64_t v = blockIdx.x; v < n; v += gridDim.x) {
        const float* yr = y + v * G.y_dim;
        float* hr = h + v * G.h_dim;
        for (int j = threadIdx.x; j < G.h_dim; j += blockDim.x) {
            if (G.last || j < G.mul0) {
                hr[j] = silu_(yr[j]);
                continue;
            }
            const int l = 1 + (G.lmax >= 2 && j >= G.h_off[2]) + (G.lmax >= 3 && j >= G.h_off[3]);
            const int r = j - irrep_sel(G.h_off, l);
            const int u = r % irrep_sel(G.mul, l);
            const float gate = silu_(yr[G.mul0 + irrep_sel(G.goff, l) + u]);
            hr[j] = yr[irrep_sel(G.y_off, l) + r] * gate;
        }
    }
}

void launch_gate_fwd(const LayerDev& L, int mul0, const int* mul, int lmax, int64_t n,
                     const float* y, float* h, cudaStream_t st) {
    const GateDims G = gate_dims(L, mul0, mul, lmax);
    if (n == 0 || G.h_dim == 0) return;
    gate_fwd_kernel<<<gate_grid(n), 256, 0, st>>>(G, n, y, h);
}

// gy = dE/dy from gh = dE/dh (or, for the last block, the readout vector)
__global__ void gate_bwd_kernel(const GateDims G, int64_t n, const float* __restrict__ y,
                                const float* __restrict__ gh, const float* __restrict__ readout,
                                float* __restrict__ gy) {
    for (int64_t v = blockIdx.x; v < n; v += gridDim.x) {
        const float* yr = y + v * G.y_dim;
        const float* ghr = gh + v * G.h_dim;
        float* gyr = gy + v * G.y_dim;
        for (int j = threadIdx.x; j < G.y_dim; j += blockDim.x) {
            if (G.last) {
                gyr[j] = readout[j] * dsilu_(yr[j]);
                continue;
            }
            if (j < G.mul0) {
                gyr[j] = ghr[j] * dsilu_(yr[j]);
                continue;
            }
            if (j < G.mul0 + G.ng) {               // a gate scalar
                const int gidx = j - G.mul0;
                const int l = 1 + (G.lmax >= 2 && gidx >= G.goff[2]) + (G.lmax >= 3 && gidx >= G.goff[3]);
                const int u = gidx - irrep_sel(G.goff, l);
                const int ml = irrep_sel(G.mul, l), ho = irrep_sel(G.h_off, l), yo = irrep_sel(G.y_off, l);
                float s = 0.0f;
                for (int mm = 0; mm < 2 * l + 1; ++mm) {
                    const int off = mm * ml + u;
                    s = fmaf(ghr[ho + off], yr[yo + off], s);
                }
                gyr[j] = s * dsilu_(yr[j]);
                continue;
            }
            const int l = 1 + (G.lmax >= 2 && j >= G.y_off[2]) + (G.lmax >= 3 && j >= G.y_off[3]);
            const int r = j - irrep_sel(G.y_off, l);
            const int u = r % irrep_sel(G.mul, l);
            gyr[j] = ghr[irrep_sel(G.h_off, l) + r] * silu_(yr[G.mul0 + irrep_sel(G.goff, l) + u]);
        }
    }
}

void launch_gate_bwd(const LayerDev& L, int mul0, const int* mul, int lmax, int64_t n,
                     const float* y, const float* gh, const float* readout, float* gy,
                     cudaStream_t st) {
    const GateDims G = gate_dims(L, mul0, mul, lmax);
    if (n == 0 || G.y_dim == 0) return;
    gate_bwd_kernel<<<gate_grid(n), 256, 0, st>>>(G, n, y, gh, readout, gy);
}

// ---------------------------------------------------------------- readout
__global__ void readout_kernel(const float* __restrict__ h, int h_dim, const float* __restrict__ c,
                               const double* __restrict__ shift, const int* __restrict__ species,
                               int64_t n, int mul0, int n_species, double* __restrict__ e_atom) {
    const int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (v >= n) return;
    float s = 0.0f;
    for (int u = lane; u < mul0; u += 32) s = fmaf(h[v * h_dim + u], c[u], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) e_atom[v] = (double)s + shift[clamp_species(species[v], n_species)];
}

void launch_readout(const float* h, int h_dim, const float* c, const double* shift,
                    const int* species, int64_t n, int mul0, int n_species, double* e_atom, cudaStream_t st) {
    if (n == 0) return;
    const int64_t threads = n * 32;
    readout_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(h, h_dim, c, shift, species,
                                                                      n, mul0, n_species, e_atom);
}

// ---------------------------------------------------------------- forces / virial
__global__ void forces_kernel(int64_t n, const int* __restrict__ row_ptr, const int* __restrict__ rev,
                              const float* __restrict__ gd, const float4* __restrict__ geom,
                              double* __restrict__ f, double* __restrict__ w) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    double fx = 0, fy = 0, fz = 0;
    double wv[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
        const float* g = gd + (int64_t)e * 3;
        const float* gr = gd + (int64_t)rev[e] * 3;
        const double g0 = g[0], g1 = g[1], g2 = g[2];
        fx += g0 - (double)gr[0];
        fy += g1 - (double)gr[1];
        fz += g2 - (double)gr[2];
        const float4 d = geom[e];
        const double dd[3] = {d.x, d.y, d.z};
        const double gg[3] = {g0, g1, g2};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) wv[a * 3 + b] -= gg[a] * dd[b];
    }
    f[v * 3 + 0] = fx;
    f[v * 3 + 1] = fy;
    f[v * 3 + 2] = fz;
#pragma unroll
    for (int k = 0; k < 9; ++k) w[v * 9 + k] = wv[k];
}

void launch_forces(int64_t n, const int* row_ptr, const int* rev, const float* gd,
                   const float4* geom, double* f_s, double* w_atom, cudaStream_t st) {
    if (n == 0) return;
    forces_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(n, row_ptr, rev, gd, geom, f_s, w_atom);
}

// One CTA per structure: fixed-order FP64 sums of atom energies and virials
// (per thread over a strided set of atoms, then a fixed shuffle tree per warp
// and over the warps), so repeated evaluations give identical sums.
constexpr int RS_THREADS = 1024;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(RS_THREADS) reduce_structs_kernel(const int64_t* __restrict__ atom_off,
                                                                    const double* __restrict__ e_atom,
                                                                    const double* __restrict__ w_atom,
                                                                    double* __restrict__ energy,
                                                                    double* __restrict__ virial) {
    const int s = blockIdx.x;
    const int64_t a0 = atom_off[s], a1 = atom_off[s + 1];
    double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll 4
    for (int64_t v = a0 + threadIdx.x; v < a1; v += RS_THREADS) {
        acc[0] += e_atom[v];
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[1 + k] += w_atom[v * 9 + k];
    }
    __shared__ double red[RS_THREADS / 32][10];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        const double w = warp_sum_d(acc[k]);
        if (lane == 0) red[warp][k] = w;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < 10; ++k) acc[k] = warp_sum_d(red[lane][k]);
        if (lane == 0) {
            if (energy) energy[s] = acc[0];
            if (virial)
                for (int k = 0; k < 9; ++k) virial[s * 9 + k] = acc[1 + k];
        }
    }
}

void launch_reduce_structs(int32_t n_structs, const int64_t* atom_off, const double* e_atom,
                           const double* w_atom, double* energy, double* virial, cudaStream_t st) {
    if (n_structs == 0) return;
    reduce_structs_kernel<<<n_structs, RS_THREADS, 0, st>>>(atom_off, e_atom, w_atom, energy, virial);
}

__global__ void scatter_forces_kernel(int64_t n, const int* __restrict__ perm,
                                      const double* __restrict__ f_s, double* __restrict__ forces) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t o = perm[i];
    forces[o * 3 + 0] = f_s[i * 3 + 0];
    forces[o * 3 + 1] = f_s[i * 3 + 1];
    forces[o * 3 + 2] = f_s[i * 3 + 2];
}

void launch_scatter_forces(int64_t n, const int* perm, const double* f_s, double* forces,
                           cudaStream_t st) {
    if (n == 0 || !forces) return;
    scatter_forces_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, perm, f_s, forces);
}

}  // namespace sn
