// Cell-list neighbour build for a batch of periodic cells (paper Sec. 2: an
// edge joins v and w when |r_w - r_v| < r_c; every periodic image counts).
//
// Steps (all on the device; the synchronous form reads the edge count back once,
// the asynchronous form keeps it on the device and relies on a preallocated
// capacity, with an overflow flag and a clamped CSR when that is too small):
//   1. fractional coordinates, wrap along periodic directions, bin index
//      (bins at least r_c wide per lattice direction, per structure);
//   2. counting sort of atoms by bin, ties broken by input index, which fixes
//      the internal (spatially sorted) atom order;
//   3. per receiver, scan the bins within the search range (more than one
//      neighbouring bin when a cell is thinner than r_c, e.g. self-images),
//      count, prefix-sum into row_ptr, then write (dst, src, shift, d, |d|);
//   4. index of the reverse edge (w, v, -S) of every edge.
// The distance test is FP64 on FP64 positions.
#include "internal.h"

namespace sn {

// per-structure descriptor (ints): [0..2] bins per direction, [3..5] search
// range, [6..8] pbc, [9] bin base, [10] atom begin, [11] atom end
constexpr int SD = 16;

__device__ __forceinline__ int struct_of_atom(const int64_t* __restrict__ atom_off, int S, int64_t i) {
    int lo = 0, hi = S;     // largest s with atom_off[s] <= i
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (atom_off[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

// cond (may be null): every kernel of the build returns at once when *cond is 0
// (the Verlet-list rebuild of MD decided on the device).
__device__ __forceinline__ bool skip(const int* cond) { return cond && *cond == 0; }

__global__ void bin_atoms_kernel(int64_t n, int S, const int64_t* __restrict__ atom_off,
                                 const int* __restrict__ sdesc, const double* __restrict__ inv_cells,
                                 const double* __restrict__ pos, int* __restrict__ bin_of,
                                 int* __restrict__ bin_count, const int* cond) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || skip(cond)) return;
    const int s = struct_of_atom(atom_off, S, i);
    const int* d = sdesc + s * SD;
    const double* ic = inv_cells + s * 9;
    const double p[3] = {pos[i * 3], pos[i * 3 + 1], pos[i * 3 + 2]};
    int b[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        // fractional coordinate a = p . column a of inv(cell)
        double f = p[0] * ic[0 * 3 + a] + p[1] * ic[1 * 3 + a] + p[2] * ic[2 * 3 + a];
        if (d[6 + a]) f -= floor(f);
        int bi = (int)floor(f * d[a]);
        bi = bi < 0 ? 0 : (bi >= d[a] ? d[a] - 1 : bi);
        b[a] = bi;
    }
    const int bin = d[9] + (b[0] * d[1] + b[1]) * d[2] + b[2];
    bin_of[i] = bin;
    atomicAdd(bin_count + bin, 1);
}

// Exclusive scan of n ints into out[0..n] (out[n] = total) with one CTA.
__global__ void __launch_bounds__(1024) scan_kernel(const int* __restrict__ in, int64_t n,
                                                    int* __restrict__ out, int* __restrict__ total,
                                                    const int* cond) {
    if (skip(cond)) return;
    __shared__ int warp_sums[32];
    __shared__ int carry;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += 1024) {
        const int64_t i = base + t;
        const int x = (i < n) ? in[i] : 0;
        int s = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane == 31) warp_sums[w] = s;
        __syncthreads();
        if (w == 0) {
            int ws = warp_sums[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, ws, o);
                if (lane >= o) ws += y;
            }
            warp_sums[lane] = ws;
        }
        __syncthreads();
        const int excl = carry + (w ? warp_sums[w - 1] : 0) + s - x;
        if (i < n) out[i] = excl;
        __syncthreads();
        if (t == 1023) carry = excl + x;
        __syncthreads();
    }
    if (t == 0) {
        out[n] = carry;
        if (total) *total = carry;
    }
}

__global__ void place_kernel(int64_t n, const int* __restrict__ bin_of, const int* __restrict__ bin_start,
                             int* __restrict__ bin_fill, int* __restrict__ perm, const int* cond) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || skip(cond)) return;
    const int b = bin_of[i];
    const int slot = atomicAdd(bin_fill + b, 1);
    perm[bin_start[b] + slot] = (int)i;
}

// Sort each bin's members by input index (deterministic internal order).
__global__ void sort_bins_kernel(int64_t n_bins, const int* __restrict__ bin_start, int* __restrict__ perm,
                                 const int* cond) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_bins || skip(cond)) return;
    const int s0 = bin_start[b], s1 = bin_start[b + 1];
    for (int i = s0 + 1; i < s1; ++i) {
        const int key = perm[i];
        int j = i - 1;
        while (j >= s0 && perm[j] > key) {
            perm[j + 1] = perm[j];
            --j;
        }
        perm[j + 1] = key;
    }
}

// Gather species into internal order, with the wrapped position q = p - n cell and
// the integer image n of every atom (n = floor of the fractional coordinate along
// periodic directions).
__global__ void gather_kernel(int64_t n, int S, const int64_t* __restrict__ atom_off,
                              const int* __restrict__ sdesc, const double* __restrict__ cells,
                              const double* __restrict__ inv_cells, const int* __restrict__ perm,
                              const double* __restrict__ pos, const int32_t* __restrict__ species,
                              double* __restrict__ pos_s, double* __restrict__ fl_s, float4* __restrict__ q32,
                              int* __restrict__ species_s, int* __restrict__ struct_of, const int* cond) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || skip(cond)) return;
    const int64_t o = perm[i];
    const int s = struct_of_atom(atom_off, S, i);
    const int* d = sdesc + s * SD;
    const double* ic = inv_cells + s * 9;
    const double p[3] = {pos[o * 3], pos[o * 3 + 1], pos[o * 3 + 2]};
    double fl[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double f = p[0] * ic[0 * 3 + a] + p[1] * ic[1 * 3 + a] + p[2] * ic[2 * 3 + a];
        fl[a] = d[6 + a] ? floor(f) : 0.0;
        fl_s[i * 3 + a] = fl[a];
    }
    const double* c = cells + s * 9;
    double q[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {     // wrapped position q = p - fl cell
        q[a] = p[a] - (fl[0] * c[0 * 3 + a] + fl[1] * c[1 * 3 + a] + fl[2] * c[2 * 3 + a]);
        pos_s[i * 3 + a] = q[a];
    }
    q32[i] = make_float4((float)q[0], (float)q[1], (float)q[2], 0.0f);
    species_s[i] = species[o];
    struct_of[i] = s;
}

// Count (FILL = false) or write (FILL = true) the edges of every internal atom
// v.  A group of NGL lanes serves one receiver: it scans the bins within the
// search range in a fixed order, the members of a bin in order, NGL candidates
// at a time; a ballot over the group gives each hit its slot, so the edge order
// is the serial one (bin order, then member order).  d = q_w - q_v + S~ cell,
// with q the wrapped positions; the edge's shift is S~ - n_w + n_v.  The test
// that decides an edge is FP64.  An FP32 pre-test skips the FP64 work for
// candidates clearly outside r_c; its margin, 1e-3 A + 1e-6 (|q_v| + |S~ cell| +
// r_c), is over ten times the FP32 rounding of d for any coordinates (positions
// along non-periodic directions are not wrapped), so it cannot drop an edge.
constexpr int NGL = 2;

__device__ __forceinline__ int floor_div(int a, int n) { return a >= 0 ? a / n : -((n - 1 - a) / n); }

template <bool FILL>
__global__ void __launch_bounds__(128)
edges_kernel(int64_t n, double rc2, float rc32, int64_t cap, const int* __restrict__ sdesc,
             const double* __restrict__ cells, const int* __restrict__ struct_of, const int* __restrict__ bin_start,
             const double* __restrict__ q_s, const float4* __restrict__ q32, const double* __restrict__ fl_s,
             const int* __restrict__ row_ptr,
             int* __restrict__ counts, int* __restrict__ flags, int* __restrict__ dst, int* __restrict__ src,
             int* __restrict__ shift, float4* __restrict__ geom, const int* cond) {
    const int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / NGL;
    if (v >= n || skip(cond)) return;                      // the whole group leaves together
    const int j = threadIdx.x & (NGL - 1);
    const int gsh = threadIdx.x & 31 & ~(NGL - 1);
    const unsigned gmask = ((1u << NGL) - 1) << gsh;
    const int s = struct_of[v];
    const int* d = sdesc + s * SD;
    const double* c = cells + s * 9;
    const double qv[3] = {q_s[v * 3], q_s[v * 3 + 1], q_s[v * 3 + 2]};
    const float4 qv32 = q32[v];
    const float qmag = fmaxf(fabsf(qv32.x), fmaxf(fabsf(qv32.y), fabsf(qv32.z)));
    float c32[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) c32[a] = (float)c[a];
    int bv[3];
    {
        const int base = d[9];
        const int nb = d[0] * d[1] * d[2];
        int lo = base, hi = base + nb;   // largest b with bin_start[b] <= v
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (bin_start[mid] <= v) lo = mid; else hi = mid;
        }
        const int local = lo - base;
        bv[2] = local % d[2];
        bv[1] = (local / d[2]) % d[1];
        bv[0] = local / (d[2] * d[1]);
    }
    int64_t e = FILL ? (int64_t)row_ptr[v] : 0;
    bool close = false;
    for (int ox = -d[3]; ox <= d[3]; ++ox) {
        int bx = bv[0] + ox, sx = 0;
        if (d[6]) { sx = floor_div(bx, d[0]); bx -= sx * d[0]; }
        else if (bx < 0 || bx >= d[0]) continue;
        for (int oy = -d[4]; oy <= d[4]; ++oy) {
            int by = bv[1] + oy, sy = 0;
            if (d[7]) { sy = floor_div(by, d[1]); by -= sy * d[1]; }
            else if (by < 0 || by >= d[1]) continue;
            for (int oz = -d[5]; oz <= d[5]; ++oz) {
                int bz = bv[2] + oz, sz = 0;
                if (d[8]) { sz = floor_div(bz, d[2]); bz -= sz * d[2]; }
                else if (bz < 0 || bz >= d[2]) continue;
                const int b = d[9] + (bx * d[1] + by) * d[2] + bz;
                const float fx = (float)sx, fy = (float)sy, fz = (float)sz;
                const float sh32[3] = {fx * c32[0] + fy * c32[3] + fz * c32[6],
                                       fx * c32[1] + fy * c32[4] + fz * c32[7],
                                       fx * c32[2] + fy * c32[5] + fz * c32[8]};
                const float smag = fmaxf(fabsf(sh32[0]), fmaxf(fabsf(sh32[1]), fabsf(sh32[2])));
                const float rpre = rc32 + 1e-3f + 1e-6f * (qmag + smag + rc32);
                const float rc2_pre = rpre * rpre;
                const int w1 = bin_start[b + 1];
                for (int w0 = bin_start[b]; w0 < w1; w0 += NGL) {
                    const int w = w0 + j;
                    bool hit = false;
                    double dd[3], r2 = 0.0;
                    if (w < w1) {
                        const float4 qw = q32[w];
                        const float ex = qw.x - qv32.x + sh32[0], ey = qw.y - qv32.y + sh32[1],
                                    ez = qw.z - qv32.z + sh32[2];
                        if (ex * ex + ey * ey + ez * ez < rc2_pre) {
                            const double sh[3] = {
                                sx * c[0] + sy * c[3] + sz * c[6],
                                sx * c[1] + sy * c[4] + sz * c[7],
                                sx * c[2] + sy * c[5] + sz * c[8]};
#pragma unroll
                            for (int a = 0; a < 3; ++a) dd[a] = q_s[w * 3 + a] - qv[a] + sh[a];
                            r2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
                            const bool self = (w == v) && sx == 0 && sy == 0 && sz == 0;
                            hit = !self && r2 < rc2;
                        }
                    }
                    const unsigned mine = (__ballot_sync(gmask, hit) >> gsh) & ((1u << NGL) - 1);
                    if constexpr (FILL) {
                        if (hit) {
                            const int64_t slot = e + __popc(mine & ((1u << j) - 1));
                            if (slot < cap) {
                                dst[slot] = (int)v;
                                src[slot] = w;
                                shift[slot * 3 + 0] = sx - (int)fl_s[w * 3 + 0] + (int)fl_s[v * 3 + 0];
                                shift[slot * 3 + 1] = sy - (int)fl_s[w * 3 + 1] + (int)fl_s[v * 3 + 1];
                                shift[slot * 3 + 2] = sz - (int)fl_s[w * 3 + 2] + (int)fl_s[v * 3 + 2];
                                geom[slot] = make_float4((float)dd[0], (float)dd[1], (float)dd[2], (float)sqrt(r2));
                            }
                        }
                    } else {
                        if (hit && r2 < 1e-16) close = true;
                    }
                    e += __popc(mine);
                }
            }
        }
    }
    if constexpr (!FILL) {
        if (j == 0) counts[v] = (int)e;
        if (close) atomicOr(flags + 1, 1);
    }
}

// Edge count over capacity: flags[0] holds the count the scan wrote.  When it
// exceeds cap, row_ptr is clamped to cap (so that no later kernel reads past
// the edge arrays), flags[FLAG_EDGE_OVERFLOW] is set and flags[FLAG_EDGE_NEED]
// keeps the largest count seen, for the caller's retry with more room.
__global__ void clamp_rows_kernel(int64_t n, int* __restrict__ row_ptr, int64_t cap, int* __restrict__ flags,
                                  const int* cond) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n || skip(cond)) return;
    const int total = flags[0];
    if ((int64_t)total <= cap) return;
    if (row_ptr[i] > cap) row_ptr[i] = (int)cap;
    if (i == 0) {
        flags[FLAG_EDGE_OVERFLOW] = 1;
        atomicMax(flags + FLAG_EDGE_NEED, total);
    }
}

// Reverse edge of every edge e < row_ptr[n] (launched over the capacity).
__global__ void reverse_kernel(int64_t n, int64_t cap, const int* __restrict__ row_ptr, const int* __restrict__ dst,
                               const int* __restrict__ src, const int* __restrict__ shift,
                               int* __restrict__ rev, int* __restrict__ flags, const int* cond) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= cap || skip(cond) || e >= row_ptr[n]) return;
    const int v = dst[e], w = src[e];
    const int s0 = -shift[e * 3], s1 = -shift[e * 3 + 1], s2 = -shift[e * 3 + 2];
    int found = -1;
    for (int k = row_ptr[w]; k < row_ptr[w + 1]; ++k) {
        if (src[k] == v && shift[k * 3] == s0 && shift[k * 3 + 1] == s1 && shift[k * 3 + 2] == s2) {
            found = k;
            break;
        }
    }
    if (found < 0) {
        atomicOr(flags + 2, 1);
        found = (int)e;
    }
    rev[e] = found;
}

// Unordered pairs: edge e stands for the pair {e, rev[e]} when e < rev[e]
// (rev[e] != e for every edge of a symmetric list, since d != 0).  A warp per
// receiver v counts (FILL = false) or writes (FILL = true) its pairs in edge
// order, so the pair list is ordered by receiver like the edges.
template <bool FILL>
__global__ void pairs_kernel(int64_t n, const int* __restrict__ row_ptr, const int* __restrict__ rev,
                             const int* __restrict__ dst, const int* __restrict__ src,
                             const float4* __restrict__ geom, int* __restrict__ cnt,
                             const int* __restrict__ pair_ptr, int* __restrict__ p_e, int* __restrict__ p_dst,
                             int* __restrict__ p_src, float4* __restrict__ p_geom) {
    const int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (v >= n) return;                                    // whole warps
    const int e0 = row_ptr[v], e1 = row_ptr[v + 1];
    int k = FILL ? pair_ptr[v] : 0;
    for (int b = e0; b < e1; b += 32) {
        const int e = b + lane;
        const bool take = e < e1 && e < rev[e];
        const unsigned m = __ballot_sync(0xffffffffu, take);
        if (FILL && take) {
            const int o = k + __popc(m & ((1u << lane) - 1u));
            p_e[o] = e;
            p_dst[o] = dst[e];
            p_src[o] = src[e];
            p_geom[o] = geom[e];
        }
        k += __popc(m);
    }
    if (!FILL && lane == 0) cnt[v] = k;
}

void build_pairs(Workspace* ws, int64_t N, cudaStream_t st) {
    const unsigned blocks = (unsigned)((std::max<int64_t>(N, 1) * 32 + 255) / 256);
    if (N > 0)
        pairs_kernel<false><<<blocks, 256, 0, st>>>(N, ws->row_ptr, ws->rev, nullptr, nullptr, nullptr, ws->row_cnt,
                                                   nullptr, nullptr, nullptr, nullptr, nullptr);
    scan_kernel<<<1, 1024, 0, st>>>(ws->row_cnt, N, ws->pair_ptr, nullptr, nullptr);
    if (N > 0)
        pairs_kernel<true><<<blocks, 256, 0, st>>>(N, ws->row_ptr, ws->rev, ws->dst, ws->src, ws->geom, nullptr,
                                                  ws->pair_ptr, ws->p_e, ws->p_dst, ws->p_src, ws->p_geom);
}

// ---------------------------------------------------------------- host side
static void cell_geometry(const double* c, double* inv, double* width, double* det_out) {
    const double det = c[0] * (c[4] * c[8] - c[5] * c[7]) - c[1] * (c[3] * c[8] - c[5] * c[6]) +
                       c[2] * (c[3] * c[7] - c[4] * c[6]);
    *det_out = det;
    inv[0] = (c[4] * c[8] - c[5] * c[7]) / det;
    inv[1] = (c[2] * c[7] - c[1] * c[8]) / det;
    inv[2] = (c[1] * c[5] - c[2] * c[4]) / det;
    inv[3] = (c[5] * c[6] - c[3] * c[8]) / det;
    inv[4] = (c[0] * c[8] - c[2] * c[6]) / det;
    inv[5] = (c[2] * c[3] - c[0] * c[5]) / det;
    inv[6] = (c[3] * c[7] - c[4] * c[6]) / det;
    inv[7] = (c[1] * c[6] - c[0] * c[7]) / det;
    inv[8] = (c[0] * c[4] - c[1] * c[3]) / det;
    // perpendicular width along lattice direction i: |det| / |a_j x a_k|
    for (int i = 0; i < 3; ++i) {
        const double* a = c + ((i + 1) % 3) * 3;
        const double* b = c + ((i + 2) % 3) * 3;
        const double cx = a[1] * b[2] - a[2] * b[1];
        const double cy = a[2] * b[0] - a[0] * b[2];
        const double cz = a[0] * b[1] - a[1] * b[0];
        width[i] = fabs(det) / sqrt(cx * cx + cy * cy + cz * cz);
    }
}

static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

sevennet_status build_neighbors(sevennet_model* M, Workspace* ws, const BatchHost& b,
                                const double* pos_dev, const int32_t* species_dev,
                                cudaStream_t st, int64_t* n_edges_out, double r_list, const int* cond,
                                bool async) {
    const int S = b.n_structs;
    const int64_t N = b.atom_off[S];
    const double rc = r_list > 0.0 ? r_list : M->cfg.r_cut;
    // per-structure bins
    std::vector<int> sdesc((size_t)S * SD, 0);
    std::vector<double> inv((size_t)S * 9);
    int64_t n_bins = 0;
    for (int s = 0; s < S; ++s) {
        double width[3], det;
        cell_geometry(&b.cells[(size_t)s * 9], &inv[(size_t)s * 9], width, &det);
        SN_CHECK(std::isfinite(det) && fabs(det) > 1e-12, SEVENNET_EINVAL,
                 "structure %d: singular cell", s);
        int* d = &sdesc[(size_t)s * SD];
        int64_t nb = 1;
        for (int a = 0; a < 3; ++a) {
            int nbin = (int)floor(width[a] / rc);
            if (nbin < 1) nbin = 1;
            if (nbin > 512) nbin = 512;
            const int pbc = b.pbc.empty() ? 1 : (b.pbc[(size_t)s * 3 + a] != 0);
            int k = (int)ceil(rc * nbin / width[a] - 1e-12);
            if (k < 1) k = 1;
            SN_CHECK(!pbc || k <= 16, SEVENNET_EINVAL,
                     "structure %d: cell thinner than r_c/16 along direction %d", s, a);
            if (!pbc) k = 1;
            d[a] = nbin;
            d[3 + a] = k;
            d[6 + a] = pbc;
            nb *= nbin;
        }
        d[9] = (int)n_bins;
        d[10] = (int)b.atom_off[s];
        d[11] = (int)b.atom_off[s + 1];
        n_bins += nb;
    }
    SN_CHECK(n_bins < (1LL << 30), SEVENNET_EINVAL, "too many cell-list bins");
    int64_t cap_e = async ? ws->cap_edges : std::max<int64_t>(ws->cap_edges, std::max<int64_t>(N * 64, 1024));
    SN_CHECK(!async || cap_e > 0, SEVENNET_EINVAL, "internal error: asynchronous build without edge capacity");
    SN_TRY(ws_reserve(M, ws, N, cap_e, n_bins, S, st));
    SN_CUDA(cudaMemcpyAsync(ws->sdesc, sdesc.data(), sdesc.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    SN_CUDA(cudaMemcpyAsync(ws->cells, b.cells.data(), (size_t)S * 9 * sizeof(double), cudaMemcpyHostToDevice, st));
    SN_CUDA(cudaMemcpyAsync(ws->inv_cells, inv.data(), (size_t)S * 9 * sizeof(double), cudaMemcpyHostToDevice, st));
    SN_CUDA(cudaMemcpyAsync(ws->atom_off, b.atom_off.data(), (size_t)(S + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    SN_CUDA(cudaMemsetAsync(ws->bin_count, 0, (size_t)(n_bins + 1) * sizeof(int), st));
    SN_CUDA(cudaMemsetAsync(ws->bin_fill, 0, (size_t)(n_bins + 1) * sizeof(int), st));
    if (!async) SN_CUDA(cudaMemsetAsync(ws->flags, 0, FLAG_WORDS * sizeof(int), st));
    if (N > 0) {
        bin_atoms_kernel<<<blocks_for(N, 256), 256, 0, st>>>(N, S, ws->atom_off, ws->sdesc, ws->inv_cells,
                                                            pos_dev, ws->bin_of, ws->bin_count, cond);
    }
    scan_kernel<<<1, 1024, 0, st>>>(ws->bin_count, n_bins, ws->bin_start, nullptr, cond);
    if (N > 0) {
        place_kernel<<<blocks_for(N, 256), 256, 0, st>>>(N, ws->bin_of, ws->bin_start, ws->bin_fill, ws->perm,
                                                        cond);
        sort_bins_kernel<<<blocks_for(n_bins, 128), 128, 0, st>>>(n_bins, ws->bin_start, ws->perm, cond);
        gather_kernel<<<blocks_for(N, 256), 256, 0, st>>>(N, S, ws->atom_off, ws->sdesc, ws->cells,
                                                         ws->inv_cells, ws->perm, pos_dev, species_dev,
                                                         ws->pos_s, ws->frac_floor, ws->q32, ws->species_s,
                                                         ws->struct_of, cond);
        edges_kernel<false><<<blocks_for(N * NGL, 128), 128, 0, st>>>(
            N, rc * rc, (float)rc, 0, ws->sdesc, ws->cells, ws->struct_of, ws->bin_start, ws->pos_s, ws->q32,
            ws->frac_floor, nullptr, ws->row_cnt, ws->flags, nullptr, nullptr, nullptr, nullptr, cond);
    }
    scan_kernel<<<1, 1024, 0, st>>>(ws->row_cnt, N, ws->row_ptr, ws->flags + 0, cond);
    int64_t E = -1;                                      // asynchronous: the count stays on the device
    if (!async) {
        SN_CUDA(cudaMemcpyAsync(ws->flags_host, ws->flags, FLAG_WORDS * sizeof(int), cudaMemcpyDeviceToHost, st));
        SN_CUDA(cudaStreamSynchronize(st));
        E = ws->flags_host[0];
        SN_CHECK(ws->flags_host[1] == 0, SEVENNET_EINVAL, "two atoms closer than 1e-8 A");
        if (E > ws->cap_edges) SN_TRY(ws_reserve(M, ws, N, E + E / 4 + 1024, n_bins, S, st));
    }
    if (N > 0) {
        edges_kernel<true><<<blocks_for(N * NGL, 128), 128, 0, st>>>(
            N, rc * rc, (float)rc, ws->cap_edges, ws->sdesc, ws->cells, ws->struct_of, ws->bin_start, ws->pos_s,
            ws->q32, ws->frac_floor, ws->row_ptr, nullptr, ws->flags, ws->dst, ws->src, ws->shift, ws->geom, cond);
        clamp_rows_kernel<<<blocks_for(N + 1, 256), 256, 0, st>>>(N, ws->row_ptr, ws->cap_edges, ws->flags, cond);
    }
    const int64_t span = async ? ws->cap_edges : E;
    if (span > 0)
        reverse_kernel<<<blocks_for(span, 256), 256, 0, st>>>(N, span, ws->row_ptr, ws->dst, ws->src, ws->shift,
                                                             ws->rev, ws->flags, cond);
    SN_CUDA(cudaGetLastError());
    *n_edges_out = E;
    return SEVENNET_OK;
}

// ---------------------------------------------------------------- Verlet list refresh
// Group of NGL lanes per receiver v over its stored list entries, in order:
// d = p_w - p_v + shift cell at the current positions (input order through perm),
// FP64; kept when |d| < r_c.  Count pass, then fill pass into the compact CSR.
template <bool FILL>
__global__ void __launch_bounds__(128)
refresh_kernel(int64_t n, double rc2, int64_t cap, const int* __restrict__ perm, const double* __restrict__ pos,
               const double* __restrict__ cell, const int* __restrict__ lrow, const int* __restrict__ lsrc,
               const int* __restrict__ lshift, const int* __restrict__ row_ptr, int* __restrict__ counts,
               int* __restrict__ dst, int* __restrict__ src, int* __restrict__ shift, float4* __restrict__ geom,
               int* __restrict__ flags, int64_t lcap) {
    const int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / NGL;
    if (v >= n) return;
    const int j = threadIdx.x & (NGL - 1);
    const int gsh = threadIdx.x & 31 & ~(NGL - 1);
    const unsigned gmask = ((1u << NGL) - 1) << gsh;
    const int64_t ov = perm[v];
    const double pv[3] = {pos[ov * 3], pos[ov * 3 + 1], pos[ov * 3 + 2]};
    int64_t e = FILL ? (int64_t)row_ptr[v] : 0;
    int k1 = lrow[v + 1];
    const int kb = lrow[v];
    if (kb < 0 || (int64_t)k1 > lcap || kb > k1) {       // rows outside the stored list: reported
        if (!FILL && j == 0) atomicOr(flags + 2, 1);
        k1 = kb;
    }
    for (int k0 = kb; k0 < k1; k0 += NGL) {
        const int k = k0 + j;
        bool hit = false;
        double dd[3], r2 = 0.0;
        int w = 0, s0 = 0, s1 = 0, s2 = 0;
        if (k < k1) w = lsrc[k];
        if (k < k1 && (w < 0 || (int64_t)w >= n)) {     // not an atom: a corrupt list, reported
            if (!FILL) atomicOr(flags + 2, 1);
            w = 0;
        } else if (k < k1) {
            s0 = lshift[k * 3]; s1 = lshift[k * 3 + 1]; s2 = lshift[k * 3 + 2];
            const int64_t ow = perm[w];
#pragma unroll
            for (int a = 0; a < 3; ++a)
                dd[a] = pos[ow * 3 + a] - pv[a] + (s0 * cell[a] + s1 * cell[3 + a] + s2 * cell[6 + a]);
            r2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
            hit = r2 < rc2;
        }
        const unsigned mine = (__ballot_sync(gmask, hit) >> gsh) & ((1u << NGL) - 1);
        if constexpr (FILL) {
            if (hit) {
                const int64_t slot = e + __popc(mine & ((1u << j) - 1));
                if (slot < cap) {
                    dst[slot] = (int)v;
                    src[slot] = w;
                    shift[slot * 3 + 0] = s0;
                    shift[slot * 3 + 1] = s1;
                    shift[slot * 3 + 2] = s2;
                    geom[slot] = make_float4((float)dd[0], (float)dd[1], (float)dd[2], (float)sqrt(r2));
                }
            }
        }
        e += __popc(mine);
    }
    if constexpr (!FILL) {
        if (j == 0) counts[v] = (int)e;
    }
}

sevennet_status refresh_neighbors(sevennet_model* M, Workspace* ws, int64_t N, const double* pos_dev,
                                  const int* list_row_ptr, const int* list_src, const int* list_shift,
                                  int64_t list_cap, cudaStream_t st, int64_t* n_edges_out) {
    // asynchronous: the count stays on the device, the arrays are sized by capacity
    const double rc = M->cfg.r_cut;
    if (N > 0)
        refresh_kernel<false><<<blocks_for(N * NGL, 128), 128, 0, st>>>(
            N, rc * rc, 0, ws->perm, pos_dev, ws->cells, list_row_ptr, list_src, list_shift, nullptr,
            ws->row_cnt, nullptr, nullptr, nullptr, nullptr, ws->flags, list_cap);
    scan_kernel<<<1, 1024, 0, st>>>(ws->row_cnt, N, ws->row_ptr, ws->flags + 0, nullptr);
    if (N > 0) {
        refresh_kernel<true><<<blocks_for(N * NGL, 128), 128, 0, st>>>(
            N, rc * rc, ws->cap_edges, ws->perm, pos_dev, ws->cells, list_row_ptr, list_src, list_shift,
            ws->row_ptr, nullptr, ws->dst, ws->src, ws->shift, ws->geom, ws->flags, list_cap);
        clamp_rows_kernel<<<blocks_for(N + 1, 256), 256, 0, st>>>(N, ws->row_ptr, ws->cap_edges, ws->flags,
                                                                 nullptr);
    }
    if (ws->cap_edges > 0)
        reverse_kernel<<<blocks_for(ws->cap_edges, 256), 256, 0, st>>>(N, ws->cap_edges, ws->row_ptr, ws->dst,
                                                                      ws->src, ws->shift, ws->rev, ws->flags,
                                                                      nullptr);
    SN_CUDA(cudaGetLastError());
    *n_edges_out = -1;
    return SEVENNET_OK;
}

}  // namespace sn
