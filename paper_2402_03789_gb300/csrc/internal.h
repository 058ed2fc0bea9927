// Internal declarations of the SevenNet GB300 library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "sevennet.h"

namespace sn {

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
extern thread_local std::string g_last_error;

#define SN_CUDA(call)                                                              \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            ::sn::set_error("%s:%d: %s: %s", __FILE__, __LINE__, #call,            \
                            cudaGetErrorString(e_));                               \
            return SEVENNET_ECUDA;                                                 \
        }                                                                          \
    } while (0)

#define SN_CHECK(cond, code, ...)                                                  \
    do {                                                                           \
        if (!(cond)) {                                                             \
            ::sn::set_error(__VA_ARGS__);                                          \
            return (code);                                                         \
        }                                                                          \
    } while (0)

// Entry of a C-ABI call: select the device and drop any error a previous,
// unrelated runtime call left behind (so it is not reported as ours).
#define SN_ENTER(dev)                                                              \
    do {                                                                           \
        cudaGetLastError();                                                        \
        SN_CUDA(cudaSetDevice(dev));                                               \
    } while (0)

#define SN_TRY(expr)                                                               \
    do {                                                                           \
        sevennet_status s_ = (expr);                                               \
        if (s_ != SEVENNET_OK) return s_;                                          \
    } while (0)

// ---------------------------------------------------------------- model
constexpr int MAX_PATHS = 40;
constexpr int CONV_THREADS = 256;
constexpr int CONV_WARPS = CONV_THREADS / 32;
constexpr int MAX_SLOTS = 12;
constexpr int EC = 16;                 // edges per chunk in the convolution kernels
// CTAs per SM of the convolution kernels: two for lmax <= 2; the lmax 3 tiles
// (34 paths) need more shared memory and registers than half an SM holds.
__host__ __device__ constexpr int conv_ctas_per_sm(int lmax) { return lmax >= 3 ? 1 : 2; }
constexpr int MAX_NB = 16;             // radial basis functions
constexpr int MAX_LMAX = 3;
constexpr int NL = MAX_LMAX + 1;     // irreps l = 0..MAX_LMAX

// kind = canonical index of the coupling (l1, l2, l3) among the 34 with l <= 3:
// the 15 with every l <= 2 first (0..14, dense for the lmax <= 2 kernels), then
// the 19 with some l = 3; within each group l1-major, then l2, then l3.
__host__ __device__ constexpr int coupling_kind(int l1, int l2, int l3) {
    int k = 0;
    for (int top = 2; top <= MAX_LMAX; ++top)
        for (int a = 0; a <= top; ++a)
            for (int b = 0; b <= top; ++b)
                for (int c = (a > b ? a - b : b - a); c <= (a + b < top ? a + b : top); ++c) {
                    if (top > 2 && a <= 2 && b <= 2 && c <= 2) continue;     // counted in the first group
                    if (a == l1 && b == l2 && c == l3) return k;
                    ++k;
                }
    return -1;
}

// Path set of a block, known at compile time from (l1, lmax, kind): the
// couplings (l1, l2, l3) with |l1-l2| <= l3 <= min(l1+l2, lmax), l2 <= lmax;
// the first block has l1 = 0 only, the last keeps l3 = 0 only.  Same order as
// the block's runtime path table.
struct PathList {
    int n;
    int l2[12];
    int l3[12];
};

__host__ __device__ constexpr PathList path_list(int l1, int lmax, int kind) {
    PathList p{0, {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0}, {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0}};
    if (((kind & 1) && l1 != 0) || l1 > lmax) return p;
    for (int l2 = 0; l2 <= lmax; ++l2)
        for (int l3 = (l1 > l2 ? l1 - l2 : l2 - l1); l3 <= (l1 + l2 < lmax ? l1 + l2 : lmax); ++l3) {
            if ((kind & 2) && l3 != 0) continue;
            p.l2[p.n] = l2;
            p.l3[p.n] = l3;
            ++p.n;
        }
    return p;
}

__host__ __device__ constexpr int path_begin(int l1, int lmax, int kind) {
    int s = 0;
    for (int l = 0; l < l1; ++l) s += path_list(l, lmax, kind).n;
    return s;
}

// Forward convolution work sets: the path list of one input irrep l1 split into
// contiguous subsets of at most fwd_set_cap(kind) multiply-adds per channel
// and edge (a path costs (2 l1 + 1)(2 l3 + 1) for x G and 2 l3 + 1 for the
// weight).  One set shares the gather of x_src[l1] over its paths; its running
// sums stay in registers.  Large sets cut gathers and code; the first block
// (scalar input only) uses small sets so that its few paths still give every
// warp work.
constexpr int FWD_MAX_SETS = 6;
__host__ __device__ constexpr int fwd_set_cap(int kind) { return (kind & 1) ? 8 : 96; }

struct PathSets {
    int n;          // number of sets
    int b[FWD_MAX_SETS + 1];   // set j holds paths [b[j], b[j + 1]) of path_list(l1, lmax, kind)
};

__host__ __device__ constexpr int fwd_path_cost(int l1, int l3) { return (2 * l1 + 1) * (2 * l3 + 1) + 2 * l3 + 1; }

__host__ __device__ constexpr PathSets fwd_path_sets(int l1, int lmax, int kind) {
    PathSets s{0, {0, 0, 0, 0, 0, 0, 0}};
    const PathList p = path_list(l1, lmax, kind);
    if (p.n == 0) return s;
    int cost = 0;
    for (int i = 0; i < p.n; ++i) {
        const int c = fwd_path_cost(l1, p.l3[i]);
        if (cost > 0 && cost + c > fwd_set_cap(kind)) {
            s.b[++s.n] = i;
            cost = 0;
        }
        cost += c;
    }
    s.b[++s.n] = p.n;
    return s;
}

// Running sums per channel of set j: sum of 2 l3 + 1 over its paths.
__host__ __device__ constexpr int fwd_set_nacc(int l1, int lmax, int kind, int j) {
    const PathList p = path_list(l1, lmax, kind);
    const PathSets s = fwd_path_sets(l1, lmax, kind);
    int n = 0;
    for (int i = s.b[j]; i < s.b[j + 1]; ++i) n += 2 * p.l3[i] + 1;
    return n;
}

__host__ __device__ constexpr int fwd_set_cost(int l1, int lmax, int kind, int j) {
    const PathList p = path_list(l1, lmax, kind);
    const PathSets s = fwd_path_sets(l1, lmax, kind);
    int n = 0;
    for (int i = s.b[j]; i < s.b[j + 1]; ++i) n += fwd_path_cost(l1, p.l3[i]);
    return n;
}

// Channels per lane (CPL) the forward kernel is compiled for: several channels
// share one G matrix and the address arithmetic.  The register budget of 2 CTAs
// per SM allows CPL (2 l1 + 1) <= 6 gathered values and CPL * nacc <= 20 running
// sums; only the H = 64 kernel carries the wider groups.
__host__ __device__ constexpr bool fwd_cpl_compiled(int H, int l1, int nacc, int cpl) {
    return cpl == 1 || (H == 64 && cpl * (2 * l1 + 1) <= 6 && cpl * nacc <= 20);
}

// Tensor-core forward (BF16 path): the contraction over (edge, m1) runs on
// mma.m16n8k16 with 16 channels as M, m3 as N and K = 16 slots holding
// (edge, m1) pairs of edges that share a receiver.  EG edges fill one K group:
// 16 for l1 = 0, 4 for l1 = 1 (3 slots each, one padding), 2 for l1 = 2, 3
// (two lanes of 4 slots per edge).  The paths of one input irrep are split
// into sets of at most 24 / (16 / EG) paths; a work unit is one set over 16
// channels.
__host__ __device__ constexpr int tc_eg(int n1) { return n1 == 1 ? 16 : (n1 == 3 ? 4 : 2); }
__host__ __device__ constexpr int tc_nkg(int n1) { return EC / tc_eg(n1); }
__host__ __device__ constexpr int tc_set_cap(int n1) { return 24 / tc_nkg(n1); }
constexpr int TC_MAX_SETS = 6;
constexpr int MAX_SLOTS_TC = 24;

__host__ __device__ constexpr PathSets tc_path_sets(int l1, int lmax, int kind) {
    PathSets s{0, {0, 0, 0, 0, 0, 0, 0}};
    const PathList p = path_list(l1, lmax, kind);
    if (p.n == 0) return s;
    const int cap = tc_set_cap(2 * l1 + 1);
    int n = 0;
    for (int i = 0; i < p.n; ++i) {
        if (n == cap) { s.b[++s.n] = i; n = 0; }
        ++n;
    }
    s.b[++s.n] = p.n;
    return s;
}

struct PathDesc {
    int32_t l1, l2, l3, kind;
    int32_t mul;      // channels of the path (= multiplicity of l1 in the block input)
    int32_t col0;     // first radial-MLP output column of the path
    int32_t x_off;    // offset of the l1 block inside an x row
    int32_t m_off;    // offset of the l3 block inside a message row
    int32_t m_mul;    // channels of the l3 message block
    int32_t m_ch0;    // first channel of this path inside the l3 block
    int32_t g_off;    // offset of this path's G matrix in the per-edge buffer
    int32_t b_off;    // tensor-core forward: first 32-bit word of the path's B fragments in shared memory
};

// Everything a convolution kernel needs to know about one block.
struct ConvDesc {
    int32_t n_paths;
    int32_t W;          // radial MLP output width (sum of path channels)
    int32_t Wpad;       // row stride (floats) of the per-edge weight tile in shared memory (FP32 tile)
    int32_t H;          // hidden width of the radial MLP
    int32_t n_basis;
    int32_t lmax;       // spherical-harmonic degree
    int32_t ys;         // floats per edge of the Y (and dE/dY) tiles: max(9, (lmax + 1)^2)
    int32_t x_dim;      // row width of x (block input after linear_1)
    int32_t m_dim;      // row width of the messages
    int32_t nG;         // floats of G per edge
    int32_t l1max;
    int32_t mul_in[NL];  // multiplicity of l in the block input (0 = absent)
    int32_t x_off[NL];
    int32_t pbeg[NL], pend[NL];   // paths with l1 = l occupy [pbeg, pend)
    int32_t kind;               // bit 0: first block (input mul0 x 0e), bit 1: last block (l3 = 0)
    float r_cut;
    float env_a, env_b, env_c;  // envelope coefficients
    int32_t poly_p;
    PathDesc paths[MAX_PATHS];
    int16_t n_slots[CONV_WARPS];
    int16_t slot_group[CONV_WARPS][MAX_SLOTS];  // (l1 << 11) | (set << 8) | (channel block << 2) | log2 CPL
    int32_t WpadB;      // row stride (BF16 values) of the BF16 weight tile: rows start on 16 bytes
    // tensor-core forward (BF16): work units, B-fragment words, staged x rows
    int16_t n_slots_tc[CONV_WARPS];
    int16_t slot_tc[CONV_WARPS][MAX_SLOTS_TC];  // (l1 << 12) | (set << 8) | 16-channel tile
    int32_t nBF;                  // 32-bit words of B fragments per chunk
    int32_t xs_off[NL];           // floats: staged x region of irrep l1 (EC rows)
    int32_t xs_stride[NL];        // floats between the staged rows of two edges
    int32_t xs_total;             // floats of the staged x regions
    int32_t tc_ok;                // 1: the block can run the tensor-core forward
};

// One row-block matrix product of a per-irrep linear: rows are (atom, m)
// pairs, row r -> atom v = r / R, component m = r % R, A row at
// A + v*lda + a_off + m*K, C row at C + v*ldc + c_off + m*N.
struct GemmProb {
    const float* A;
    const float* B;            // [K][N] row-major FP32 (pre-scaled)
    const __nv_bfloat16* Bh;   // [N][K] BF16 transpose (hi), followed by the lo term at Bh + K*N
    float* C;
    int64_t n_atoms;
    int32_t R, K, N;           // K and N are multiples of 32 (every multiplicity is)
    int32_t lda, a_off, ldc, c_off;
    int32_t accumulate;        // 1: C += A B, 0: C = A B
};
constexpr int MAX_GEMM_PROBS = 8;
struct GemmBatch {
    int32_t n;
    GemmProb p[MAX_GEMM_PROBS];
};

struct LayerDev {
    ConvDesc conv;
    int x_dim, y_dim, h_in_dim, h_out_dim, m_dim;
    int in_mul[NL], y_mul[NL], msg_mul[NL], out_mul[NL];
    int in_off[NL], y_off[NL], msg_off[NL], out_off[NL];
    bool last;
    // device weights, pre-scaled by 1/sqrt(fan_in) (and 1/avg_num_neigh for mlp2)
    float* mlp0 = nullptr;   // [NB][H]
    float* mlp1 = nullptr;   // [H][H]
    float* mlp2 = nullptr;   // [H][W]
    float* mlp0T = nullptr;  // [H][NB]
    float* mlp1T = nullptr;  // [H][H]
    float* mlp2T = nullptr;  // [W][H]
    __nv_bfloat16* mlp1h = nullptr;   // [2][H][H] W2 as stored, hi then lo (B operand of gA2 @ W2^T)
    __nv_bfloat16* mlp1Th = nullptr;  // [2][H][H] W2^T, hi then lo (B operand of H1 @ W2)
    __nv_bfloat16* mlp2h = nullptr;   // [W][H]  (N-major for mma B operand)
    __nv_bfloat16* mlp2Th = nullptr;  // [H][W]
    float* lin1[NL] = {};  float* lin1T[NL] = {};  __nv_bfloat16* lin1h[NL] = {};  __nv_bfloat16* lin1Th[NL] = {};
    float* sc[NL] = {};    float* scT[NL] = {};    __nv_bfloat16* sch[NL] = {};    __nv_bfloat16* scTh[NL] = {};
    float* lin2[NL] = {};  float* lin2T[NL] = {};  __nv_bfloat16* lin2h[NL] = {};  __nv_bfloat16* lin2Th[NL] = {};
};

struct Workspace;

// Kernel-family timing with CUDA events (diagnostics).
enum ProfFamily { PF_NEIGHBORS = 0, PF_LINEAR, PF_CONV_FWD, PF_CONV_BWD, PF_GATE, PF_OTHER, PF_COUNT };
struct Profiler {
    bool on = false;
    struct Rec { int fam; cudaEvent_t a, b; };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    double total_ms[PF_COUNT] = {0};
    int64_t launches[PF_COUNT] = {0};
    cudaEvent_t get();
};
void prof_begin(Profiler* p, int fam, cudaStream_t st, cudaEvent_t* a);
void prof_end(Profiler* p, int fam, cudaStream_t st, cudaEvent_t a, int n_launches);
void count_launches(int n);

}  // namespace sn

struct sevennet_model {
    int device = 0;
    sevennet_model_config cfg{};
    std::vector<double> shift;
    int T = 0, lmax = 0, H = 0, NB = 0;
    int h_max = 0, x_max = 0, y_max = 0, m_max = 0;
    std::vector<sn::LayerDev> layers;
    float* embed = nullptr;     // [n_species][mul0]
    float* readout = nullptr;   // [mul0] = scale * R0 R1 / sqrt(mul0 hid)
    double* shift_dev = nullptr;
    cudaStream_t stream = nullptr;
    sn::Workspace* ws = nullptr;
    sn::Profiler prof;
    std::vector<void*> allocations;
};

namespace sn {

// ---------------------------------------------------------------- workspace
struct Workspace {
    int64_t cap_atoms = 0, cap_edges = 0, cap_bins = 0, cap_structs = 0;
    // neighbour build (internal atom order = cell-sorted)
    int* bin_of = nullptr;        // [N] bin of each input atom
    int* bin_count = nullptr;     // [bins+1]
    int* bin_start = nullptr;     // [bins+1]
    int* bin_fill = nullptr;      // [bins]
    int* perm = nullptr;          // [N] internal -> input index
    int* struct_of = nullptr;     // [N] internal atom -> structure
    double* pos_s = nullptr;      // [N][3] wrapped positions in internal order
    double* frac_floor = nullptr; // [N][3] integer image of each internal atom
    float4* q32 = nullptr;        // [N] wrapped positions in FP32 (distance pre-test)
    int* species_s = nullptr;     // [N]
    int* row_ptr = nullptr;       // [N+1]
    int* row_cnt = nullptr;       // [N+1]
    int* dst = nullptr;           // [E]
    int* src = nullptr;           // [E]
    int* shift = nullptr;         // [E][3]
    int* rev = nullptr;           // [E]
    float4* geom = nullptr;       // [E] (d, r)
    // unordered pairs {e, rev[e]} with e < rev[e], in receiver order (the adjoint's units)
    int* pair_ptr = nullptr;      // [N+1] pairs of receivers < v; pair_ptr[N] = number of pairs
    int* p_e = nullptr;           // [E] edge of each pair
    int* p_dst = nullptr;         // [E] its receiver
    int* p_src = nullptr;         // [E] its sender
    float4* p_geom = nullptr;     // [E] its (d, r)
    // per-structure descriptors (device)
    double* cells = nullptr;      // [S][9]
    double* inv_cells = nullptr;  // [S][9]
    int* sdesc = nullptr;         // [S][16] bins, offsets, search ranges, pbc
    int64_t* atom_off = nullptr;  // [S+1]
    // model activations
    float* h = nullptr;           // [N][h_max]
    float* xs = nullptr;          // [T][N][x_max]
    float* ys = nullptr;          // [T][N][y_max]
    float* m = nullptr;           // [N][m_max] (messages, then their gradients)
    float* gy = nullptr;          // [N][y_max]
    float* gx = nullptr;          // [N][x_max]
    unsigned long long* gxq = nullptr;   // [N][x_max] fixed-point sums of dE/dx
    float* gh = nullptr;          // [N][h_max]
    float* gd = nullptr;          // [E][3]
    double* e_atom = nullptr;     // [N]
    double* w_atom = nullptr;     // [N][9]
    double* f_s = nullptr;        // [N][3] forces, internal order
    int* flags = nullptr;         // [FLAG_WORDS] device status words
    int* flags_host = nullptr;    // pinned mirror
    std::vector<void*> allocs;
};

// host helpers implemented in the .cu files
sevennet_status ws_reserve(sevennet_model* M, Workspace* ws, int64_t n_atoms, int64_t n_edges,
                           int64_t n_bins, int64_t n_structs, cudaStream_t st);
void ws_free(Workspace* ws);

struct BatchHost {
    int32_t n_structs;
    std::vector<int64_t> atom_off;   // [S+1]
    std::vector<double> cells;       // [S][9]
    std::vector<int32_t> pbc;        // [S][3]
};

// Neighbour build for a batch; positions/species are device arrays in input
// order.  Leaves ws->row_ptr/src/dst/shift/geom/rev and the internal order.
// r_list > 0 builds the list for that cutoff instead of the model's r_c (the
// Verlet list of MD with a skin).
// async: no host synchronisation (the caller has reserved the edge capacity and
// cleared the flags; *n_edges_out = -1 and the count stays on the device);
// cond (device int, may be null): every kernel skips when *cond is 0.
sevennet_status build_neighbors(sevennet_model* M, Workspace* ws, const BatchHost& b,
                                const double* pos_dev, const int32_t* species_dev,
                                cudaStream_t st, int64_t* n_edges_out, double r_list = 0.0,
                                const int* cond = nullptr, bool async = false);

// The edges of a stored Verlet list (CSR in the internal order of the build that
// made it: row_ptr, src, shift) that are within the model's r_c at the current
// positions (input order), kept in list order, into ws->row_ptr/src/dst/shift/
// geom/rev.  One structure; the internal order and cell of that build stay valid.
// Asynchronous (*n_edges_out = -1; the count stays on the device).  list_cap is
// the number of entries the list arrays hold: a row beyond it or a sender that
// is not an atom is skipped and sets flags[2].
sevennet_status refresh_neighbors(sevennet_model* M, Workspace* ws, int64_t n_atoms, const double* pos_dev,
                                  const int* list_row_ptr, const int* list_src, const int* list_shift,
                                  int64_t list_cap, cudaStream_t st, int64_t* n_edges_out);

// The steps of run_model, for callers that interleave work between blocks
// (the domain-decomposed evaluation): all operate on the N atoms and E edges of
// the workspace's graph.
void model_embed(sevennet_model* M, Workspace* ws, int64_t N, cudaStream_t st);
void model_layer_forward(sevennet_model* M, Workspace* ws, int t, int64_t N, int64_t E,
                         sevennet_precision prec, cudaStream_t st);
void model_readout(sevennet_model* M, Workspace* ws, int64_t N, cudaStream_t st);
void model_layer_backward_gate(sevennet_model* M, Workspace* ws, int t, int64_t N, cudaStream_t st);
// pairs: the convolution adjoint runs over ws's pair list (built by build_pairs
// from a symmetric neighbour list); otherwise per edge.
sevennet_status model_layer_backward_rest(sevennet_model* M, Workspace* ws, int t, int64_t N, int64_t E,
                                          sevennet_precision prec, cudaStream_t st, bool pairs = false);

// Model evaluation on the internal order prepared by build_neighbors.
sevennet_status run_model(sevennet_model* M, Workspace* ws, const BatchHost& b, int64_t n_edges,
                          sevennet_precision prec, double* energy_dev, double* forces_dev,
                          double* virial_dev, cudaStream_t st);

// Device status words of a workspace: [0] edge count of the last build or
// refresh, [1] two atoms closer than 1e-8 A, [2] reverse edge missing, [3]
// species out of range, [FLAG_GX_OVERFLOW], [FLAG_EDGE_OVERFLOW] edges beyond
// the capacity, [FLAG_EDGE_NEED] the largest edge count asked for,
// [FLAG_COPY_TIMEOUT] a bulk copy not completed within its bounded wait.
constexpr int FLAG_WORDS = 8;
constexpr int FLAG_EDGE_OVERFLOW = 4;
constexpr int FLAG_EDGE_NEED = 6;
constexpr int FLAG_COPY_TIMEOUT = 7;     // a bounded wait for a bulk copy ran out

// Deterministic scatter of dE/dx in the convolution adjoint: every per-edge
// contribution v is added as the 64-bit integer round(v * 2^36) (fixed point),
// so the sums are the same whatever order the atomics land in.  A contribution
// that is not finite or has |v| >= GX_LIMIT adds GX_SENTINEL instead and sets
// flags[FLAG_GX_OVERFLOW]; a sum of magnitude >= 2^56 converts to NaN.
constexpr float GX_SCALE = 68719476736.0f;          // 2^36
constexpr float GX_LIMIT = 65536.0f;                // 2^16
constexpr long long GX_SENTINEL = 1LL << 57;
constexpr int FLAG_GX_OVERFLOW = 5;

// kernels launchers (conv.cu / node.cu)
// flags (may be null) receives FLAG_COPY_TIMEOUT from the tensor-core forward
void launch_conv_fwd(const LayerDev& L, int H, sevennet_precision prec, int64_t n_atoms,
                     int64_t n_edges, const int* row_ptr, const int* dst, const int* src,
                     const float4* geom, const float* x, float* m, cudaStream_t st, int* flags = nullptr);
// n_edges is an upper bound on the edge count (the count itself is read from
// row_ptr[n_atoms] on the device); gxq is an [n_atoms][x_dim] 64-bit scratch for
// the fixed-point sums of dE/dx; gx == nullptr skips them (the first block's
// input gradient is not needed) and flags (may be null) receives the overflow flag.
void launch_conv_bwd(const LayerDev& L, int H, sevennet_precision prec, int64_t n_atoms,
                     int64_t n_edges, const int* row_ptr, const int* dst, const int* src,
                     const float4* geom, const float* x, const float* gm, float* gx,
                     unsigned long long* gxq, int* flags, float* gd, cudaStream_t st);
sevennet_status conv_configure(int H, const std::vector<LayerDev>& layers);
// tensor-core forward of the BF16 path (conv_fwd_tc.cu)
size_t conv_tc_smem_bytes(const ConvDesc& D, int H);
sevennet_status conv_configure_fwd_tc(int H, size_t need);
void launch_conv_fwd_tc(const LayerDev& L, int H, int64_t n_atoms, int64_t n_edges, const int* row_ptr,
                        const int* dst, const int* src, const float4* geom, const float* x, float* m,
                        int* flags, cudaStream_t st);
void launch_gemm(const GemmBatch& b, sevennet_precision prec, cudaStream_t st);
// The adjoint over unordered pairs (ws->pair_ptr / p_*): n_pairs is an upper
// bound on the pair count (the count is pair_ptr[n_atoms], on the device); the
// pair's whole dE/dd goes to its edge p_e, the reverse edge's entry is left as is.
void launch_conv_bwd_pair(const LayerDev& L, int H, sevennet_precision prec, int64_t n_atoms, int64_t n_pairs,
                          const int* pair_ptr, const int* p_dst, const int* p_src, const float4* p_geom,
                          const int* p_e, const float* x, const float* gm, float* gx, unsigned long long* gxq,
                          int* flags, float* gd, cudaStream_t st);
void launch_gx_from_fixed(size_t nx, const unsigned long long* gxq, float* gx, int* flags, cudaStream_t st);
// The pair list of the current neighbour list (needs row_ptr, rev, dst, src, geom).
void build_pairs(Workspace* ws, int64_t N, cudaStream_t st);
void launch_embed(const float* table, const int* species, int64_t n, int mul0, int n_species, float* h,
                  cudaStream_t st);
void launch_gate_fwd(const LayerDev& L, int mul0, const int* mul, int lmax, int64_t n,
                     const float* y, float* h, cudaStream_t st);
void launch_gate_bwd(const LayerDev& L, int mul0, const int* mul, int lmax, int64_t n,
                     const float* y, const float* gh, const float* readout, float* gy,
                     cudaStream_t st);
void launch_readout(const float* h, int h_dim, const float* c, const double* shift,
                    const int* species, int64_t n, int mul0, int n_species, double* e_atom, cudaStream_t st);
void launch_forces(int64_t n, const int* row_ptr, const int* rev, const float* gd,
                   const float4* geom, double* f_s, double* w_atom, cudaStream_t st);
void launch_reduce_structs(int32_t n_structs, const int64_t* atom_off, const double* e_atom,
                           const double* w_atom, double* energy, double* virial, cudaStream_t st);
void launch_scatter_forces(int64_t n, const int* perm, const double* f_s, double* forces,
                           cudaStream_t st);

int num_sms(int device);

// dst and (d, |d|) of caller-provided CSR edges (conv entry points)
void conv_prepare_edges(int64_t n_atoms, int64_t n_edges, const int* row_ptr, const float* d,
                        int* dst, float4* geom, cudaStream_t st);

// shared by the C ABI front ends (api.cu, md_server.cu)
sevennet_status eval_enqueue(sevennet_model* M, Workspace* ws, const BatchHost& b,
                             const int32_t* species_dev, const double* pos_dev, sevennet_precision prec,
                             double* energy_dev, double* forces_dev, double* virial_dev, cudaStream_t st);
sevennet_status check_flags(const int* flags_host);
void reserve_edges(sevennet_model* M, Workspace* ws, int64_t N, int64_t need, sevennet_status* s);
sevennet_status eval_batch(sevennet_model* M, Workspace* ws, const BatchHost& b,
                           const int32_t* species_dev, const double* pos_dev,
                           sevennet_precision prec, double* energy_dev, double* forces_dev,
                           double* virial_dev, cudaStream_t st);
sevennet_status check_batch(const BatchHost& b);

}  // namespace sn
