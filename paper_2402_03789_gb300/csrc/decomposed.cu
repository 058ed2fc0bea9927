// Single-process emulation of the paper's spatial decomposition (Sec. 3.1,
// Figure 3): the cell is cut into slabs along the first lattice vector; each
// domain owns the atoms of its slab and keeps ghost copies of every atom that
// sends an edge to one of its own atoms (a shell one r_c deep, not r_c times
// the number of layers).  Per block, each domain updates only its own atoms:
//   forward  - after the block, every ghost copy of h is refreshed from its
//              owner (the forward exchange of Figure 3c-d);
//   adjoint  - before the adjoint of a block, the dE/dh that a domain's edges
//              left on its ghosts is added to the owners and cleared (the
//              reverse exchange of Figure 3e); a domain's energy counts its own
//              atoms only, so its ghosts take no readout gradient;
//   forces   - every edge adds +dE/dd to its receiver and -dE/dd to its sender
//              (Eq. 6), straight into the global force array (the reverse
//              exchange of partial forces, Figure 3f); the virial sums
//              -dE/dd (x) d over all edges of all domains.
// The exchanges go through device buffers indexed by global atom.  The result
// equals the single-domain evaluation up to FP summation order, and repeats
// bit for bit: the sums that several domains or edges add into (ghost
// gradients, forces) are 64-bit fixed point, and the virial's per-block
// partials are added in block order.
#include "internal.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace sn {

// glob[gid[i]] = loc[i] (rows of w floats)
__global__ void dd_put_rows(int64_t n, int w, const int* __restrict__ gid, const float* __restrict__ loc,
                            float* __restrict__ glob) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * w) return;
    const int64_t r = i / w;
    glob[(int64_t)gid[r] * w + (i % w)] = loc[i];
}

// loc[i] = glob[gid[i]]
__global__ void dd_get_rows(int64_t n, int w, const int* __restrict__ gid, const float* __restrict__ glob,
                            float* __restrict__ loc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * w) return;
    const int64_t r = i / w;
    loc[i] = glob[(int64_t)gid[r] * w + (i % w)];
}

// glob[gid[i]] += loc[i] in 64-bit fixed point (units of 2^-36; several domains
// may hold the same ghost, and integer sums do not depend on the order of the
// adds); a value that is not finite or has |v| >= 2^16 adds a sentinel instead.
__global__ void dd_push_grad(int64_t n, int w, const int* __restrict__ gid, const float* __restrict__ loc,
                             unsigned long long* __restrict__ glob) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * w) return;
    const int64_t r = i / w;
    const float v = loc[i];
    const long long q = fabsf(v) < GX_LIMIT ? __float2ll_rn(v * GX_SCALE) : GX_SENTINEL;
    atomicAdd(glob + (int64_t)gid[r] * w + (i % w), (unsigned long long)q);
}

// loc[i] += glob[gid[i]] (a sum that received the sentinel gives NaN)
__global__ void dd_pull_grad(int64_t n, int w, const int* __restrict__ gid, const unsigned long long* __restrict__ glob,
                             float* __restrict__ loc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * w) return;
    const int64_t r = i / w;
    const long long q = (long long)glob[(int64_t)gid[r] * w + (i % w)];
    const long long lim = 1LL << 56;
    loc[i] += (q >= lim || q <= -lim) ? __int_as_float(0x7fc00000) : (float)((double)q * (1.0 / 68719476736.0));
}

// Force contributions in 64-bit fixed point (units of 2^-36 eV/A); a value
// that is not finite or has |v| >= 2^26 adds a sentinel, which gives NaN.
constexpr double DD_F_LIMIT = 67108864.0;
__device__ __forceinline__ void dd_force_add(unsigned long long* p, double v) {
    const long long q = fabs(v) < DD_F_LIMIT ? __double2ll_rn(v * 68719476736.0) : GX_SENTINEL;
    atomicAdd(p, (unsigned long long)q);
}

// Edge e (receiver v <- sender w): F[v] += g_e, F[w] -= g_e (fixed point); the
// block's sum of -g_e (x) d_e goes to the partials Wp[blockIdx.x][9].
__global__ void dd_forces(int64_t E, const int* __restrict__ dst, const int* __restrict__ src,
                          const int* __restrict__ gid, const float* __restrict__ gd,
                          const float4* __restrict__ geom, unsigned long long* __restrict__ Fq,
                          double* __restrict__ Wp) {
    __shared__ double red[9][256];
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double wv[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (e < E) {
        const double g[3] = {gd[e * 3], gd[e * 3 + 1], gd[e * 3 + 2]};
        const float4 d4 = geom[e];
        const double d[3] = {d4.x, d4.y, d4.z};
        const int64_t v = gid[dst[e]], w = gid[src[e]];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            dd_force_add(Fq + v * 3 + a, g[a]);
            dd_force_add(Fq + w * 3 + a, -g[a]);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) wv[a * 3 + b] = -g[a] * d[b];
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) red[k][threadIdx.x] = wv[k];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
#pragma unroll
            for (int k = 0; k < 9; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 9) Wp[(int64_t)blockIdx.x * 9 + threadIdx.x] = red[threadIdx.x][0];
}

// F from its fixed-point sums; W = the nb block partials added in block order.
__global__ void dd_forces_out(int64_t n, const unsigned long long* __restrict__ Fq, double* __restrict__ F,
                              int64_t nb, const double* __restrict__ Wp, double* __restrict__ W) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 3 * n) {
        const long long q = (long long)Fq[i];
        const long long lim = 1LL << 56;
        F[i] = (q >= lim || q <= -lim) ? __longlong_as_double(0x7ff8000000000000LL) : (double)q * (1.0 / 68719476736.0);
    }
    if (i < 9) {
        double s = 0.0;
        for (int64_t b = 0; b < nb; ++b) s += Wp[b * 9 + i];
        W[i] = s;
    }
}

static inline unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

struct Domain {
    Workspace* ws = nullptr;
    int64_t n_own = 0, n_loc = 0, E = 0;
    int* gid = nullptr;             // [n_loc] global atom of each local atom (own first, then ghosts)
};

}  // namespace sn

using namespace sn;

extern "C" sevennet_status sevennet_eval_decomposed(sevennet_model* M, int64_t n_atoms, const int32_t* species,
                                                   const double* pos, const double* cell, int32_t n_domains,
                                                   sevennet_precision prec, double* energy, double* forces,
                                                   double* virial) {
    SN_CHECK(M && species && pos && cell && energy && n_atoms > 0, SEVENNET_EINVAL, "bad argument");
    SN_CHECK(n_domains >= 1 && n_domains <= 64, SEVENNET_EINVAL, "n_domains must be in [1, 64]");
    SN_CHECK(prec == SEVENNET_FP32 || prec == SEVENNET_BF16, SEVENNET_EINVAL, "unknown precision");
    for (int64_t i = 0; i < n_atoms; ++i)
        SN_CHECK(species[i] >= 0 && species[i] < M->cfg.n_species, SEVENNET_EINVAL, "species index out of range");
    SN_ENTER(M->device);
    // global neighbour list (input indices; per receiver in the library's order)
    sevennet_nlist* nl = nullptr;
    int64_t EG = 0;
    const int32_t pbc[3] = {1, 1, 1};
    SN_TRY(sevennet_build_neighbors(M, n_atoms, pos, cell, pbc, &nl, &EG));
    std::vector<int32_t> gdst(std::max<int64_t>(EG, 1)), gsrc(std::max<int64_t>(EG, 1));
    std::vector<int32_t> gsh((size_t)std::max<int64_t>(EG, 1) * 3);
    sevennet_status s = sevennet_nlist_export(nl, gdst.data(), gsrc.data(), gsh.data());
    sevennet_nlist_destroy(nl);
    SN_TRY(s);
    // slab of every atom along the first lattice vector (fractional coordinate, wrapped)
    const double* c = cell;
    const double det = c[0] * (c[4] * c[8] - c[5] * c[7]) - c[1] * (c[3] * c[8] - c[5] * c[6]) +
                       c[2] * (c[3] * c[7] - c[4] * c[6]);
    SN_CHECK(std::isfinite(det) && std::fabs(det) > 1e-12, SEVENNET_EINVAL, "singular cell");
    const double inv0[3] = {(c[4] * c[8] - c[5] * c[7]) / det, (c[5] * c[6] - c[3] * c[8]) / det,
                            (c[3] * c[7] - c[4] * c[6]) / det};   // first column of inv(cell)
    std::vector<int> dom(n_atoms);
    for (int64_t i = 0; i < n_atoms; ++i) {
        double f = pos[i * 3] * inv0[0] + pos[i * 3 + 1] * inv0[1] + pos[i * 3 + 2] * inv0[2];
        f -= std::floor(f);
        dom[i] = std::min(n_domains - 1, (int)(f * n_domains));
    }
    // local graphs: own atoms in receiver order of the global list, then ghosts
    std::vector<Domain> D(n_domains);
    std::vector<std::vector<int>> own(n_domains), ghost(n_domains);
    std::vector<int> seen_own(n_atoms, 0);
    for (int64_t e = 0; e < EG; ++e) {
        const int v = gdst[e];
        if (!seen_own[v]) { seen_own[v] = 1; own[dom[v]].push_back(v); }
    }
    for (int64_t i = 0; i < n_atoms; ++i)      // atoms without edges
        if (!seen_own[i]) own[dom[i]].push_back((int)i);
    sevennet_status status = SEVENNET_OK;
    float *gbuf = nullptr;
    unsigned long long *gq = nullptr, *Fq = nullptr;
    double *F = nullptr, *W = nullptr, *Wp = nullptr;
    const cudaStream_t st = M->stream;
    auto cleanup = [&]() {
        for (auto& d : D) {
            if (d.ws) ws_free(d.ws);
            cudaFree(d.gid);
        }
        cudaFree(gbuf);
        cudaFree(gq);
        cudaFree(Fq);
        cudaFree(F);
        cudaFree(W);
        cudaFree(Wp);
    };
    std::vector<int> loc(n_atoms, -1);
    for (int d = 0; d < n_domains && status == SEVENNET_OK; ++d) {
        Domain& Dm = D[d];
        std::fill(loc.begin(), loc.end(), -1);
        for (size_t k = 0; k < own[d].size(); ++k) loc[own[d][k]] = (int)k;
        // edges of own receivers, grouped by receiver in own order
        std::vector<std::vector<int64_t>> rows(own[d].size());
        for (int64_t e = 0; e < EG; ++e)
            if (dom[gdst[e]] == d) rows[loc[gdst[e]]].push_back(e);
        std::vector<int> ids = own[d];
        for (const auto& r : rows)
            for (int64_t e : r) {
                const int w = gsrc[e];
                if (loc[w] < 0) { loc[w] = (int)ids.size(); ids.push_back(w); ghost[d].push_back(w); }
            }
        Dm.n_own = (int64_t)own[d].size();
        Dm.n_loc = (int64_t)ids.size();
        std::vector<int> row_ptr(Dm.n_loc + 1, 0), ldst, lsrc;
        std::vector<float4> geo;
        std::vector<int32_t> lsp(Dm.n_loc);
        for (int64_t k = 0; k < Dm.n_loc; ++k) lsp[k] = species[ids[k]];
        for (int64_t k = 0; k < Dm.n_own; ++k) {
            for (int64_t e : rows[k]) {
                const int v = gdst[e], w = gsrc[e];
                double dd[3];
                for (int a = 0; a < 3; ++a)
                    dd[a] = pos[(int64_t)w * 3 + a] - pos[(int64_t)v * 3 + a] +
                            (gsh[e * 3] * c[a] + gsh[e * 3 + 1] * c[3 + a] + gsh[e * 3 + 2] * c[6 + a]);
                ldst.push_back((int)k);
                lsrc.push_back(loc[w]);
                geo.push_back(make_float4((float)dd[0], (float)dd[1], (float)dd[2],
                                          (float)std::sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2])));
            }
            row_ptr[k + 1] = (int)ldst.size();
        }
        for (int64_t k = Dm.n_own; k < Dm.n_loc; ++k) row_ptr[k + 1] = row_ptr[k];
        Dm.E = (int64_t)ldst.size();
        Dm.ws = new Workspace();
        status = ws_reserve(M, Dm.ws, Dm.n_loc, std::max<int64_t>(Dm.E, 1), 1, 1, st);
        if (status) break;
        if (cudaMalloc(&Dm.gid, Dm.n_loc * sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMalloc failed for a domain");
            status = SEVENNET_ENOMEM;
            break;
        }
        Workspace* ws = Dm.ws;
        if (cudaMemcpyAsync(Dm.gid, ids.data(), Dm.n_loc * sizeof(int), cudaMemcpyHostToDevice, st) ||
            cudaMemcpyAsync(ws->row_ptr, row_ptr.data(), (Dm.n_loc + 1) * sizeof(int), cudaMemcpyHostToDevice, st) ||
            cudaMemcpyAsync(ws->species_s, lsp.data(), Dm.n_loc * sizeof(int32_t), cudaMemcpyHostToDevice, st) ||
            (Dm.E > 0 &&
             (cudaMemcpyAsync(ws->dst, ldst.data(), Dm.E * sizeof(int), cudaMemcpyHostToDevice, st) ||
              cudaMemcpyAsync(ws->src, lsrc.data(), Dm.E * sizeof(int), cudaMemcpyHostToDevice, st) ||
              cudaMemcpyAsync(ws->geom, geo.data(), Dm.E * sizeof(float4), cudaMemcpyHostToDevice, st))) ||
            cudaStreamSynchronize(st)) {
            set_error("copy of a domain's graph failed");
            status = SEVENNET_ECUDA;
            break;
        }
    }
    const int T = M->T;
    int64_t wmax = 0;
    for (int t = 0; t < T; ++t) wmax = std::max<int64_t>(wmax, std::max(M->layers[t].h_in_dim, M->layers[t].h_out_dim));
    int64_t n_part = 0;                          // virial partials: one per block of dd_forces
    for (auto& d : D) n_part += d.E > 0 ? nblk(d.E) : 0;
    if (status == SEVENNET_OK &&
        (cudaMalloc(&gbuf, (size_t)n_atoms * wmax * sizeof(float)) != cudaSuccess ||
         cudaMalloc(&gq, (size_t)n_atoms * wmax * sizeof(unsigned long long)) != cudaSuccess ||
         cudaMalloc(&Fq, (size_t)n_atoms * 3 * sizeof(unsigned long long)) != cudaSuccess ||
         cudaMalloc(&F, (size_t)n_atoms * 3 * sizeof(double)) != cudaSuccess ||
         cudaMalloc(&W, 9 * sizeof(double)) != cudaSuccess ||
         cudaMalloc(&Wp, (size_t)std::max<int64_t>(n_part, 1) * 9 * sizeof(double)) != cudaSuccess)) {
        cudaGetLastError();
        set_error("cudaMalloc failed for the exchange buffers");
        status = SEVENNET_ENOMEM;
    }
    if (status) { cleanup(); return status; }
    // forward: blocks in lockstep over the domains, exchange after each block
    for (auto& d : D) model_embed(M, d.ws, d.n_loc, st);
    for (int t = 0; t < T; ++t) {
        for (auto& d : D) model_layer_forward(M, d.ws, t, d.n_loc, d.E, prec, st);
        const int w = M->layers[t].h_out_dim;
        for (auto& d : D)
            if (d.n_own) dd_put_rows<<<nblk(d.n_own * w), 256, 0, st>>>(d.n_own, w, d.gid, d.ws->h, gbuf);
        for (auto& d : D)
            if (d.n_loc > d.n_own)
                dd_get_rows<<<nblk((d.n_loc - d.n_own) * w), 256, 0, st>>>(
                    d.n_loc - d.n_own, w, d.gid + d.n_own, gbuf, d.ws->h + d.n_own * w);
    }
    for (auto& d : D) model_readout(M, d.ws, d.n_loc, st);
    // adjoint
    for (auto& d : D)
        if (d.E > 0 && cudaMemsetAsync(d.ws->gd, 0, (size_t)d.E * 3 * sizeof(float), st)) status = SEVENNET_ECUDA;
    for (int t = T - 1; t >= 0 && status == SEVENNET_OK; --t) {
        const int w = M->layers[t].h_out_dim;
        if (t < T - 1) {      // reverse exchange of dE/dh left on ghosts
            SN_CUDA(cudaMemsetAsync(gq, 0, (size_t)n_atoms * w * sizeof(unsigned long long), st));
            for (auto& d : D)
                if (d.n_loc > d.n_own)
                    dd_push_grad<<<nblk((d.n_loc - d.n_own) * w), 256, 0, st>>>(
                        d.n_loc - d.n_own, w, d.gid + d.n_own, d.ws->gh + d.n_own * w, gq);
            for (auto& d : D) {
                if (d.n_own) dd_pull_grad<<<nblk(d.n_own * w), 256, 0, st>>>(d.n_own, w, d.gid, gq, d.ws->gh);
                if (d.n_loc > d.n_own)
                    SN_CUDA(cudaMemsetAsync(d.ws->gh + d.n_own * w, 0, (size_t)(d.n_loc - d.n_own) * w * sizeof(float),
                                            st));
            }
        }
        const int yd = M->layers[t].y_dim;
        for (auto& d : D) {
            model_layer_backward_gate(M, d.ws, t, d.n_loc, st);
            if (t == T - 1 && d.n_loc > d.n_own)       // ghosts' energies belong to their owners
                SN_CUDA(cudaMemsetAsync(d.ws->gy + d.n_own * yd, 0, (size_t)(d.n_loc - d.n_own) * yd * sizeof(float),
                                        st));
            status = model_layer_backward_rest(M, d.ws, t, d.n_loc, d.E, prec, st);
            if (status) break;
        }
    }
    if (status) { cleanup(); return status; }
    // forces, virial, energy
    SN_CUDA(cudaMemsetAsync(Fq, 0, (size_t)n_atoms * 3 * sizeof(unsigned long long), st));
    int64_t part = 0;
    for (auto& d : D)
        if (d.E > 0) {
            dd_forces<<<nblk(d.E), 256, 0, st>>>(d.E, d.ws->dst, d.ws->src, d.gid, d.ws->gd, d.ws->geom, Fq,
                                                 Wp + part * 9);
            part += nblk(d.E);
        }
    dd_forces_out<<<nblk(std::max<int64_t>(3 * n_atoms, 9)), 256, 0, st>>>(n_atoms, Fq, F, part, Wp, W);
    double e_sum = 0.0;
    std::vector<double> ea;
    for (auto& d : D) {
        ea.resize(std::max<int64_t>(d.n_own, 1));
        if (d.n_own) SN_CUDA(cudaMemcpyAsync(ea.data(), d.ws->e_atom, d.n_own * sizeof(double), cudaMemcpyDeviceToHost, st));
        SN_CUDA(cudaStreamSynchronize(st));
        for (int64_t k = 0; k < d.n_own; ++k) e_sum += ea[k];
    }
    *energy = e_sum;
    if (forces) SN_CUDA(cudaMemcpyAsync(forces, F, (size_t)n_atoms * 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (virial) SN_CUDA(cudaMemcpyAsync(virial, W, 9 * sizeof(double), cudaMemcpyDeviceToHost, st));
    SN_CUDA(cudaStreamSynchronize(st));
    cleanup();
    return SEVENNET_OK;
}
