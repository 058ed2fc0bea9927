// Molecular dynamics (NVE velocity Verlet, FP64 on the device) and the
// continuous-batching evaluation server.
//
// The paper drives its potential from LAMMPS (Sec. 3.2; NVT runs in Sec. 4 and
// the melt-quench of Sec. 5.2); here the integrator is a pair of device kernels
// around the evaluation so that positions, velocities and neighbour lists never
// leave the GPU between steps.
#include "internal.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

namespace sn {

constexpr double ACC_CONV = 9.64853321e-3;   // (eV / A / amu) -> A / fs^2
constexpr double KB_EV = 8.617333262e-5;      // eV / K

__global__ void kick_drift_kernel(int64_t n, double dt, const double* __restrict__ inv_m,
                                  const double* __restrict__ f, double* __restrict__ v,
                                  double* __restrict__ x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * 3) return;
    const double vi = v[i] + 0.5 * dt * f[i] * inv_m[i / 3];
    v[i] = vi;
    x[i] += dt * vi;
}

__global__ void kick_kernel(int64_t n, double dt, const double* __restrict__ inv_m,
                            const double* __restrict__ f, double* __restrict__ v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * 3) return;
    v[i] += 0.5 * dt * f[i] * inv_m[i / 3];
}

// E_kin = 1/2 sum m v^2 in eV (one CTA, fixed order) and E_pot copied to the logs.
__global__ void energies_kernel(int64_t n, const double* __restrict__ inv_m, const double* __restrict__ v,
                                const double* __restrict__ epot, double* __restrict__ ekin_log,
                                double* __restrict__ epot_log) {
    __shared__ double red[1024];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double m = ACC_CONV / inv_m[i];       // amu
        s += m * (v[i * 3] * v[i * 3] + v[i * 3 + 1] * v[i * 3 + 1] + v[i * 3 + 2] * v[i * 3 + 2]);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *ekin_log = 0.5 * red[0] / ACC_CONV;
        *epot_log = *epot;
    }
}

// Half of the Nose-Hoover splitting over time h (one CTA, fixed reduction order):
//   xi += h/2 G;  v *= exp(-xi h);  eta += xi h;  xi += h/2 G,
// G = (2 K - N_f k_B T0) / Q, K the kinetic energy at the current velocities
// (after the scaling K becomes s^2 K exactly).  nh = {xi, eta}.
__global__ void nh_half_kernel(int64_t n, double h, const double* __restrict__ inv_m, double* __restrict__ v,
                               double* __restrict__ nh, double nf_kt0, double q) {
    __shared__ double red[1024];
    __shared__ double scale;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double m = ACC_CONV / inv_m[i];
        s += m * (v[i * 3] * v[i * 3] + v[i * 3 + 1] * v[i * 3 + 1] + v[i * 3 + 2] * v[i * 3 + 2]);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double k = 0.5 * red[0] / ACC_CONV;
        double xi = nh[0] + 0.5 * h * (2.0 * k - nf_kt0) / q;
        const double f = exp(-xi * h);
        const double eta = nh[1] + xi * h;
        xi += 0.5 * h * (2.0 * k * f * f - nf_kt0) / q;
        nh[0] = xi;
        nh[1] = eta;
        scale = f;
    }
    __syncthreads();
    const double f = scale;
    for (int64_t i = threadIdx.x; i < n * 3; i += blockDim.x) v[i] *= f;
}

// Largest squared displacement since the list was built, as the bit pattern of
// a non-negative double (ordered like the value).
__global__ void max_disp_kernel(int64_t n, const double* __restrict__ pos, const double* __restrict__ ref,
                                unsigned long long* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double d2 = 0.0;
    if (i < n) {
        const double dx = pos[i * 3] - ref[i * 3], dy = pos[i * 3 + 1] - ref[i * 3 + 1],
                     dz = pos[i * 3 + 2] - ref[i * 3 + 2];
        d2 = dx * dx + dy * dy + dz * dz;
    }
    for (int o = 16; o > 0; o >>= 1) d2 = fmax(d2, __shfl_xor_sync(0xffffffffu, d2, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(d2));
}

// The rebuild decision of the Verlet list, on the device: cond = 1 when some
// atom has moved more than half the skin since the list's build (or force is
// set); the displacement maximum is cleared for the next step and the build
// counter advanced.
__global__ void rebuild_decision_kernel(unsigned long long* __restrict__ dmax, double thr2, int force,
                                        int* __restrict__ cond, long long* __restrict__ builds) {
    const double d2 = __longlong_as_double((long long)*dmax);
    const int c = force || !(d2 <= thr2);
    *cond = c;
    *dmax = 0ull;
    if (c) *builds += 1;
}

// Keep the freshly built list (cutoff r_c + skin) and the positions it was built
// at, when cond is set: row_ptr [n + 1], src and shift [row_ptr[n]].
__global__ void keep_list_kernel(int64_t n, int64_t cap, const int* __restrict__ cond,
                                 const int* __restrict__ row_ptr, const int* __restrict__ src,
                                 const int* __restrict__ shift, const double* __restrict__ pos,
                                 int* __restrict__ l_row, int* __restrict__ l_src, int* __restrict__ l_shift,
                                 double* __restrict__ ref) {
    if (!*cond) return;
    const int64_t total = row_ptr[n];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += (int64_t)gridDim.x * blockDim.x) {
        if (i <= n) l_row[i] = row_ptr[i];
        if (i < 3 * n) ref[i] = pos[i];
        if (i < total) {
            l_src[i] = src[i];
            l_shift[i * 3] = shift[i * 3];
            l_shift[i * 3 + 1] = shift[i * 3 + 1];
            l_shift[i * 3 + 2] = shift[i * 3 + 2];
        }
    }
}

}  // namespace sn

using namespace sn;

struct sevennet_md {
    sevennet_model* M = nullptr;
    Workspace* ws = nullptr;
    cudaStream_t st = nullptr;
    int64_t N = 0;
    BatchHost b;
    sevennet_precision prec = SEVENNET_FP32;
    int32_t* species = nullptr;
    double *pos = nullptr, *vel = nullptr, *f = nullptr, *inv_m = nullptr, *ev = nullptr;
    double *ekin = nullptr, *epot = nullptr;
    int64_t log_cap = 0;
    // Verlet list (skin > 0): CSR in the internal order of its build, positions then
    double skin = 0.0;
    int *l_row = nullptr, *l_src = nullptr, *l_shift = nullptr;
    int64_t l_cap = 0;
    double* ref = nullptr;
    unsigned long long* dmax = nullptr;
    int* cond = nullptr;                 // device: rebuild the list this step
    long long* builds = nullptr;         // device: list builds so far
    bool have_list = false;
    // state at the start of the current md_step call (restored for a retry)
    double *pos0 = nullptr, *vel0 = nullptr, *f0 = nullptr, *nh0 = nullptr;
    long long* builds0 = nullptr;
    // Nose-Hoover thermostat (tau > 0): {xi, eta} on the device
    double nh_T0 = 0.0, nh_tau = 0.0;
    // linear ramp of the target from nh_T0 to nh_T1 over nh_ramp steps (0: none);
    // nh_done steps of it have run
    double nh_T1 = 0.0;
    int64_t nh_ramp = 0, nh_done = 0;
    double* nh = nullptr;
    int64_t n_builds = 0, n_edges = 0;
};

// Room for the edge lists of this MD run: the evaluation's own list and, with
// a skin, the Verlet list (cutoff r_c + skin), each at least `need` edges.
static sevennet_status md_reserve(sevennet_md* md, int64_t need) {
    sevennet_status s;
    reserve_edges(md->M, md->ws, md->N, need, &s);
    SN_TRY(s);
    const int64_t cap = md->ws->cap_edges;
    if (md->skin > 0.0 && cap > md->l_cap) {
        cudaFree(md->l_src);
        cudaFree(md->l_shift);
        md->l_src = md->l_shift = nullptr;
        md->l_cap = 0;
        md->have_list = false;                     // the stored list is gone: the next step builds one
        if (cudaMalloc(&md->l_src, cap * sizeof(int)) || cudaMalloc(&md->l_shift, cap * 3 * sizeof(int))) {
            cudaGetLastError();
            set_error("cudaMalloc failed for the Verlet list");
            return SEVENNET_ENOMEM;
        }
        md->l_cap = cap;
    }
    if (md->skin > 0.0 && !md->l_row && cudaMalloc(&md->l_row, (md->N + 1) * sizeof(int))) {
        cudaGetLastError();
        set_error("cudaMalloc failed for the Verlet list");
        return SEVENNET_ENOMEM;
    }
    return SEVENNET_OK;
}

// Forces at the current positions, enqueued without a host synchronisation.
// Without a skin: a full neighbour build and evaluation.  With a skin: the
// stored Verlet list (cutoff r_c + skin) is rebuilt when some atom has moved
// more than skin / 2 since its build (decided on the device), and otherwise
// filtered to r < r_c at the current positions (no pair can have entered r_c).
static sevennet_status md_evaluate(sevennet_md* md) {
    sevennet_model* M = md->M;
    if (md->skin <= 0.0) {
        SN_TRY(eval_enqueue(M, md->ws, md->b, md->species, md->pos, md->prec, md->ev, md->f, md->ev + 1, md->st));
        ++md->n_builds;
        return SEVENNET_OK;
    }
    const int64_t N = md->N;
    max_disp_kernel<<<(unsigned)((N + 255) / 256), 256, 0, md->st>>>(N, md->pos, md->ref, md->dmax);
    rebuild_decision_kernel<<<1, 1, 0, md->st>>>(md->dmax, 0.25 * md->skin * md->skin, md->have_list ? 0 : 1,
                                                 md->cond, md->builds);
    int64_t E = -1;
    SN_TRY(build_neighbors(M, md->ws, md->b, md->pos, md->species, md->st, &E, M->cfg.r_cut + md->skin,
                           md->cond, true));
    keep_list_kernel<<<(unsigned)std::min<int64_t>((md->l_cap + 255) / 256 + 1, 4096), 256, 0, md->st>>>(
        N, std::max<int64_t>(md->l_cap, 3 * N + 1), md->cond, md->ws->row_ptr, md->ws->src, md->ws->shift, md->pos,
        md->l_row, md->l_src, md->l_shift, md->ref);
    md->have_list = true;
    SN_TRY(refresh_neighbors(M, md->ws, N, md->pos, md->l_row, md->l_src, md->l_shift, md->l_cap, md->st, &E));
    return run_model(M, md->ws, md->b, -1, md->prec, md->ev, md->f, md->ev + 1, md->st);
}

extern "C" {

void sevennet_md_destroy(sevennet_md* md) {
    if (!md) return;
    cudaSetDevice(md->M->device);
    if (md->st) cudaStreamSynchronize(md->st);
    cudaFree(md->species);
    cudaFree(md->pos);
    cudaFree(md->vel);
    cudaFree(md->f);
    cudaFree(md->inv_m);
    cudaFree(md->ev);
    cudaFree(md->ekin);
    cudaFree(md->epot);
    cudaFree(md->l_row);
    cudaFree(md->l_src);
    cudaFree(md->l_shift);
    cudaFree(md->ref);
    cudaFree(md->dmax);
    cudaFree(md->nh);
    cudaFree(md->cond);
    cudaFree(md->builds);
    cudaFree(md->pos0);
    cudaFree(md->vel0);
    cudaFree(md->f0);
    cudaFree(md->nh0);
    cudaFree(md->builds0);
    ws_free(md->ws);
    if (md->st) cudaStreamDestroy(md->st);
    delete md;
}

sevennet_status sevennet_md_create(sevennet_model* M, int64_t n_atoms, const int32_t* species, const double* pos,
                                   const double* vel, const double* masses, const double* cell,
                                   sevennet_precision prec, sevennet_md** out) {
    SN_CHECK(M && out && species && pos && vel && masses && cell && n_atoms > 0, SEVENNET_EINVAL, "bad argument");
    *out = nullptr;
    SN_ENTER(M->device);
    for (int s = 0; s < M->cfg.n_species; ++s)
        SN_CHECK(masses[s] > 0 && std::isfinite(masses[s]), SEVENNET_EINVAL, "mass of species %d not positive", s);
    for (int64_t i = 0; i < n_atoms; ++i)
        SN_CHECK(species[i] >= 0 && species[i] < M->cfg.n_species, SEVENNET_EINVAL, "species index out of range");
    auto* md = new sevennet_md();
    md->M = M;
    md->N = n_atoms;
    md->prec = prec;
    md->b.n_structs = 1;
    md->b.atom_off = {0, n_atoms};
    md->b.cells.assign(cell, cell + 9);
    md->b.pbc = {1, 1, 1};
    md->ws = new Workspace();
    auto fail = [&](sevennet_status s) { sevennet_md_destroy(md); return s; };
    if (cudaStreamCreateWithFlags(&md->st, cudaStreamNonBlocking) != cudaSuccess) {
        set_error("cudaStreamCreate failed");
        return fail(SEVENNET_ECUDA);
    }
    std::vector<double> inv(n_atoms);
    for (int64_t i = 0; i < n_atoms; ++i) inv[i] = ACC_CONV / masses[species[i]];
    const size_t n3 = (size_t)n_atoms * 3 * sizeof(double);
    if (cudaMalloc(&md->species, n_atoms * sizeof(int32_t)) || cudaMalloc(&md->pos, n3) ||
        cudaMalloc(&md->vel, n3) || cudaMalloc(&md->f, n3) || cudaMalloc(&md->inv_m, n_atoms * sizeof(double)) ||
        cudaMalloc(&md->ev, 16 * sizeof(double)) || cudaMalloc(&md->ref, n3) ||
        cudaMalloc(&md->dmax, sizeof(unsigned long long)) || cudaMalloc(&md->nh, 2 * sizeof(double)) ||
        cudaMalloc(&md->cond, sizeof(int)) || cudaMalloc(&md->builds, sizeof(long long)) ||
        cudaMalloc(&md->pos0, n3) || cudaMalloc(&md->vel0, n3) || cudaMalloc(&md->f0, n3) ||
        cudaMalloc(&md->nh0, 2 * sizeof(double)) || cudaMalloc(&md->builds0, sizeof(long long))) {
        cudaGetLastError();
        set_error("cudaMalloc failed for MD state");
        return fail(SEVENNET_ENOMEM);
    }
    if (cudaMemcpy(md->species, species, n_atoms * sizeof(int32_t), cudaMemcpyHostToDevice) ||
        cudaMemcpy(md->pos, pos, n3, cudaMemcpyHostToDevice) || cudaMemcpy(md->vel, vel, n3, cudaMemcpyHostToDevice) ||
        cudaMemcpy(md->inv_m, inv.data(), n_atoms * sizeof(double), cudaMemcpyHostToDevice)) {
        set_error("copy of MD state failed");
        return fail(SEVENNET_ECUDA);
    }
    if (cudaMemset(md->nh, 0, 2 * sizeof(double)) || cudaMemset(md->dmax, 0, sizeof(unsigned long long)) ||
        cudaMemset(md->builds, 0, sizeof(long long))) {
        set_error("cudaMemset failed");
        return fail(SEVENNET_ECUDA);
    }
    sevennet_status s = eval_batch(M, md->ws, md->b, md->species, md->pos, prec, md->ev, md->f, md->ev + 1, md->st);
    if (s) return fail(s);
    md->n_builds = 1;
    md->n_edges = md->ws->flags_host[0];
    *out = md;
    return SEVENNET_OK;
}

// One call runs n_steps steps without a host synchronisation (the neighbour
// lists keep their edge counts on the device) and synchronises once at the end.
// An edge list that outgrew its capacity is reported by the device; the call
// then restores the state it started from, enlarges the capacity and runs again.
static sevennet_status md_run(sevennet_md* md, int64_t n_steps, double dt_fs, bool retry) {
    const int64_t n3 = md->N * 3;
    const unsigned blocks = (unsigned)((n3 + 255) / 256);
    const bool nvt = md->nh_tau > 0.0;
    const size_t b3 = (size_t)n3 * sizeof(double);
    SN_CUDA(cudaMemcpyAsync(md->pos0, md->pos, b3, cudaMemcpyDeviceToDevice, md->st));
    SN_CUDA(cudaMemcpyAsync(md->vel0, md->vel, b3, cudaMemcpyDeviceToDevice, md->st));
    SN_CUDA(cudaMemcpyAsync(md->f0, md->f, b3, cudaMemcpyDeviceToDevice, md->st));
    SN_CUDA(cudaMemcpyAsync(md->nh0, md->nh, 2 * sizeof(double), cudaMemcpyDeviceToDevice, md->st));
    SN_CUDA(cudaMemcpyAsync(md->builds0, md->builds, sizeof(long long), cudaMemcpyDeviceToDevice, md->st));
    const int64_t nh_done0 = md->nh_done, builds0 = md->n_builds;
    SN_CUDA(cudaMemsetAsync(md->ws->flags, 0, FLAG_WORDS * sizeof(int), md->st));
    for (int64_t k = 0; k < n_steps; ++k) {
        // target of this step: the ramp's value at the middle of the step, then its end value
        double t0 = md->nh_T0;
        if (md->nh_ramp > 0) {
            const double x = std::min((double)md->nh_done + 0.5, (double)md->nh_ramp) / (double)md->nh_ramp;
            t0 = md->nh_T0 + (md->nh_T1 - md->nh_T0) * x;
            if (md->nh_done < md->nh_ramp) ++md->nh_done;
        }
        const double nf_kt0 = (3.0 * md->N - 3.0) * KB_EV * t0;
        const double q = nf_kt0 * md->nh_tau * md->nh_tau;
        if (nvt) nh_half_kernel<<<1, 1024, 0, md->st>>>(md->N, 0.5 * dt_fs, md->inv_m, md->vel, md->nh, nf_kt0, q);
        kick_drift_kernel<<<blocks, 256, 0, md->st>>>(md->N, dt_fs, md->inv_m, md->f, md->vel, md->pos);
        SN_TRY(md_evaluate(md));
        kick_kernel<<<blocks, 256, 0, md->st>>>(md->N, dt_fs, md->inv_m, md->f, md->vel);
        if (nvt) nh_half_kernel<<<1, 1024, 0, md->st>>>(md->N, 0.5 * dt_fs, md->inv_m, md->vel, md->nh, nf_kt0, q);
        energies_kernel<<<1, 1024, 0, md->st>>>(md->N, md->inv_m, md->vel, md->ev, md->ekin + k, md->epot + k);
    }
    SN_CUDA(cudaGetLastError());
    long long builds = 0;
    SN_CUDA(cudaMemcpyAsync(md->ws->flags_host, md->ws->flags, FLAG_WORDS * sizeof(int), cudaMemcpyDeviceToHost,
                            md->st));
    SN_CUDA(cudaMemcpyAsync(&builds, md->builds, sizeof(long long), cudaMemcpyDeviceToHost, md->st));
    SN_CUDA(cudaStreamSynchronize(md->st));
    const int* fl = md->ws->flags_host;
    if (fl[FLAG_EDGE_OVERFLOW] && retry) {
        const int64_t need = fl[FLAG_EDGE_NEED];
        SN_CUDA(cudaMemcpyAsync(md->pos, md->pos0, b3, cudaMemcpyDeviceToDevice, md->st));
        SN_CUDA(cudaMemcpyAsync(md->vel, md->vel0, b3, cudaMemcpyDeviceToDevice, md->st));
        SN_CUDA(cudaMemcpyAsync(md->f, md->f0, b3, cudaMemcpyDeviceToDevice, md->st));
        SN_CUDA(cudaMemcpyAsync(md->nh, md->nh0, 2 * sizeof(double), cudaMemcpyDeviceToDevice, md->st));
        SN_CUDA(cudaMemcpyAsync(md->builds, md->builds0, sizeof(long long), cudaMemcpyDeviceToDevice, md->st));
        SN_CUDA(cudaStreamSynchronize(md->st));
        md->have_list = false;                      // the list arrays are reallocated
        md->nh_done = nh_done0;
        md->n_builds = builds0;
        SN_TRY(md_reserve(md, need));
        return md_run(md, n_steps, dt_fs, false);
    }
    SN_TRY(check_flags(fl));
    if (md->skin > 0.0) md->n_builds = 1 + builds;
    md->n_edges = fl[0];
    return SEVENNET_OK;
}

sevennet_status sevennet_md_step(sevennet_md* md, int64_t n_steps, double dt_fs, double* epot_log,
                                 double* ekin_log) {
    SN_CHECK(md && n_steps >= 0 && std::isfinite(dt_fs), SEVENNET_EINVAL, "bad argument");
    SN_ENTER(md->M->device);
    if (n_steps > md->log_cap) {
        cudaFree(md->ekin);
        cudaFree(md->epot);
        md->ekin = md->epot = nullptr;
        if (cudaMalloc(&md->ekin, n_steps * sizeof(double)) || cudaMalloc(&md->epot, n_steps * sizeof(double))) {
            cudaGetLastError();
            md->log_cap = 0;
            set_error("cudaMalloc failed for MD logs");
            return SEVENNET_ENOMEM;
        }
        md->log_cap = n_steps;
    }
    if (n_steps == 0) return SEVENNET_OK;
    // edge capacity: the first evaluation's count with room for density
    // fluctuations and, with a skin, for the longer Verlet list
    const double grow = md->skin > 0.0 ? std::pow((md->M->cfg.r_cut + md->skin) / md->M->cfg.r_cut, 3.0) : 1.0;
    SN_TRY(md_reserve(md, (int64_t)(1.2 * grow * (double)std::max<int64_t>(md->n_edges, 0))));
    SN_TRY(md_run(md, n_steps, dt_fs, true));
    if (epot_log) SN_CUDA(cudaMemcpy(epot_log, md->epot, n_steps * sizeof(double), cudaMemcpyDeviceToHost));
    if (ekin_log) SN_CUDA(cudaMemcpy(ekin_log, md->ekin, n_steps * sizeof(double), cudaMemcpyDeviceToHost));
    return SEVENNET_OK;
}

sevennet_status sevennet_md_get_state(const sevennet_md* md, double* pos, double* vel, double* forces) {
    SN_CHECK(md, SEVENNET_EINVAL, "NULL md");
    SN_ENTER(md->M->device);
    SN_CUDA(cudaStreamSynchronize(md->st));
    const size_t n3 = (size_t)md->N * 3 * sizeof(double);
    if (pos) SN_CUDA(cudaMemcpy(pos, md->pos, n3, cudaMemcpyDeviceToHost));
    if (vel) SN_CUDA(cudaMemcpy(vel, md->vel, n3, cudaMemcpyDeviceToHost));
    if (forces) SN_CUDA(cudaMemcpy(forces, md->f, n3, cudaMemcpyDeviceToHost));
    return SEVENNET_OK;
}

sevennet_status sevennet_md_set_skin(sevennet_md* md, double skin_A) {
    SN_CHECK(md && std::isfinite(skin_A) && skin_A >= 0.0, SEVENNET_EINVAL, "skin must be finite and >= 0");
    md->skin = skin_A;
    md->have_list = false;             // the next step builds a list for the new skin
    return SEVENNET_OK;
}

sevennet_status sevennet_md_set_nose_hoover(sevennet_md* md, double temperature_K, double tau_fs) {
    SN_CHECK(md && std::isfinite(temperature_K) && std::isfinite(tau_fs), SEVENNET_EINVAL, "bad argument");
    SN_CHECK(tau_fs <= 0.0 || temperature_K > 0.0, SEVENNET_EINVAL, "target temperature must be > 0");
    SN_CHECK(md->N >= 2, SEVENNET_EINVAL, "a thermostat needs at least two atoms");
    md->nh_T0 = temperature_K;
    md->nh_T1 = temperature_K;
    md->nh_ramp = md->nh_done = 0;
    md->nh_tau = tau_fs > 0.0 ? tau_fs : 0.0;
    return SEVENNET_OK;
}

sevennet_status sevennet_md_set_nose_hoover_ramp(sevennet_md* md, double t_start_K, double t_end_K,
                                                 int64_t n_steps, double tau_fs) {
    SN_CHECK(md && std::isfinite(t_start_K) && std::isfinite(t_end_K) && std::isfinite(tau_fs), SEVENNET_EINVAL,
             "bad argument");
    SN_CHECK(tau_fs > 0.0 && t_start_K > 0.0 && t_end_K > 0.0 && n_steps >= 1, SEVENNET_EINVAL,
             "a ramp needs tau > 0, temperatures > 0 and at least one step");
    SN_CHECK(md->N >= 2, SEVENNET_EINVAL, "a thermostat needs at least two atoms");
    md->nh_T0 = t_start_K;
    md->nh_T1 = t_end_K;
    md->nh_ramp = n_steps;
    md->nh_done = 0;
    md->nh_tau = tau_fs;
    return SEVENNET_OK;
}

sevennet_status sevennet_md_get_nose_hoover(const sevennet_md* md, double* xi, double* eta) {
    SN_CHECK(md, SEVENNET_EINVAL, "NULL md");
    SN_ENTER(md->M->device);
    double h[2];
    SN_CUDA(cudaStreamSynchronize(md->st));
    SN_CUDA(cudaMemcpy(h, md->nh, sizeof(h), cudaMemcpyDeviceToHost));
    if (xi) *xi = h[0];
    if (eta) *eta = h[1];
    return SEVENNET_OK;
}

sevennet_status sevennet_md_get_stats(const sevennet_md* md, int64_t* n_builds, int64_t* n_edges) {
    SN_CHECK(md, SEVENNET_EINVAL, "NULL md");
    if (n_builds) *n_builds = md->n_builds;
    if (n_edges) *n_edges = md->n_edges;
    return SEVENNET_OK;
}

}  // extern "C"

// ======================================================================= serving
namespace sn {

struct SrvReq {
    uint64_t ticket;
    int64_t n;
    std::vector<int32_t> species;
    std::vector<double> pos;
    double cell[9];
    double submit_s;
    size_t bytes;
};

struct SrvRes {
    bool done = false;
    sevennet_status status = SEVENNET_OK;
    double energy = 0, virial[9] = {0};
    std::vector<double> forces;
    double submit_s = 0, start_s = 0, done_s = 0;
    int32_t batch_id = -1, batch_structs = 0;
};

struct SrvSlot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    Workspace* ws = nullptr;
    bool busy = false;
    std::vector<SrvReq> reqs;
    std::vector<int64_t> off;
    BatchHost batch;
    int* h_flags = nullptr;
    size_t bytes = 0;
    int32_t batch_id = -1;
    double start_s = 0;
    int64_t cap_atoms = 0;
    int32_t cap_structs = 0;
    double *pos = nullptr, *forces = nullptr, *energy = nullptr, *virial = nullptr;
    int32_t* species = nullptr;
    double *h_pos = nullptr, *h_forces = nullptr, *h_energy = nullptr, *h_virial = nullptr;
    int32_t* h_species = nullptr;
};

}  // namespace sn

struct sevennet_server {
    sevennet_model* M = nullptr;
    size_t budget = 0;
    size_t in_flight = 0;
    int32_t max_structs = 64;
    sevennet_precision prec = SEVENNET_FP32;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<sn::SrvReq> queue;
    std::unordered_map<uint64_t, sn::SrvRes> results;
    std::vector<sn::SrvSlot> slots;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    int32_t next_batch = 0;
    int64_t slot_atoms = 0;              // atoms one slot (one batch) can hold
    std::chrono::steady_clock::time_point t0;
};

namespace sn {

static double srv_now(const sevennet_server* s) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

// Device bytes per atom of a slot's workspace: the activations of every block,
// the messages and gradients, the fixed-point dE/dx sums, and 64 edges.
static size_t bytes_per_atom(const sevennet_model* M) {
    const size_t act = (size_t)(M->T * (M->x_max + M->y_max) + M->m_max + M->y_max + M->x_max + 2 * M->h_max) *
                           sizeof(float) + (size_t)M->x_max * sizeof(unsigned long long) + 200;
    // dst, src, rev, the clamp's row entries, shift, geometry, dE/dd; the pair list (edge, dst, src, geometry)
    const size_t per_edge = 4 * 4 + 12 + 16 + 12 + 3 * 4 + 16;
    return act + per_edge * 64;
}

// Predicted device bytes of one request (its share of a slot's workspace).
static size_t predict_bytes(const sevennet_model* M, int64_t n) { return bytes_per_atom(M) * (size_t)n + 4096; }

// A slot's workspace and pinned buffers are allocated once, at server creation,
// for cap_atoms atoms (its share of the HBM budget), so that running a batch
// neither allocates nor frees (either would wait for the whole device).
static sevennet_status slot_alloc(sevennet_model* M, SrvSlot& sl, int64_t atoms, int32_t structs) {
    const int64_t A = std::max<int64_t>(atoms, 1);
    if (cudaMalloc(&sl.pos, A * 3 * sizeof(double)) || cudaMalloc(&sl.forces, A * 3 * sizeof(double)) ||
        cudaMalloc(&sl.species, A * sizeof(int32_t)) || cudaMallocHost(&sl.h_pos, A * 3 * sizeof(double)) ||
        cudaMallocHost(&sl.h_forces, A * 3 * sizeof(double)) || cudaMallocHost(&sl.h_species, A * sizeof(int32_t)) ||
        cudaMalloc(&sl.energy, structs * sizeof(double)) || cudaMalloc(&sl.virial, structs * 9 * sizeof(double)) ||
        cudaMallocHost(&sl.h_energy, structs * sizeof(double)) ||
        cudaMallocHost(&sl.h_virial, structs * 9 * sizeof(double)) ||
        cudaMallocHost(&sl.h_flags, FLAG_WORDS * sizeof(int))) {
        cudaGetLastError();
        set_error("server: allocation of %lld atoms per slot failed", (long long)A);
        return SEVENNET_ENOMEM;
    }
    sl.cap_atoms = A;
    sl.cap_structs = structs;
    // workspace: atoms, 64 edges per atom, cell-list bins and structure descriptors
    return ws_reserve(M, sl.ws, A, std::max<int64_t>(A * 64, 1024), A + 128 * (int64_t)structs, structs, sl.st);
}

// Enqueue one packed batch on a slot: copies, neighbour build and evaluation with
// the edge count kept on the device, results and status words back into pinned
// memory, an event at the end.  No host synchronisation, no allocation.
static sevennet_status slot_launch(sevennet_server* S, SrvSlot& sl) {
    const int32_t ns = (int32_t)sl.reqs.size();
    sl.start_s = srv_now(S);
    BatchHost b;
    b.n_structs = ns;
    b.atom_off.assign(ns + 1, 0);
    b.cells.resize((size_t)ns * 9);
    b.pbc.assign((size_t)ns * 3, 1);
    for (int32_t i = 0; i < ns; ++i) {
        b.atom_off[i + 1] = b.atom_off[i] + sl.reqs[i].n;
        std::copy(sl.reqs[i].cell, sl.reqs[i].cell + 9, &b.cells[(size_t)i * 9]);
    }
    const int64_t N = b.atom_off[ns];
    SN_CHECK(N <= sl.cap_atoms && ns <= sl.cap_structs, SEVENNET_ECUDA, "internal error: batch exceeds its slot");
    for (int32_t i = 0; i < ns; ++i) {
        std::copy(sl.reqs[i].pos.begin(), sl.reqs[i].pos.end(), sl.h_pos + b.atom_off[i] * 3);
        std::copy(sl.reqs[i].species.begin(), sl.reqs[i].species.end(), sl.h_species + b.atom_off[i]);
    }
    SN_TRY(check_batch(b));
    SN_CUDA(cudaMemcpyAsync(sl.pos, sl.h_pos, N * 3 * sizeof(double), cudaMemcpyHostToDevice, sl.st));
    SN_CUDA(cudaMemcpyAsync(sl.species, sl.h_species, N * sizeof(int32_t), cudaMemcpyHostToDevice, sl.st));
    SN_CUDA(cudaMemsetAsync(sl.ws->flags, 0, FLAG_WORDS * sizeof(int), sl.st));
    SN_TRY(eval_enqueue(S->M, sl.ws, b, sl.species, sl.pos, S->prec, sl.energy, sl.forces, sl.virial, sl.st));
    SN_CUDA(cudaMemcpyAsync(sl.h_energy, sl.energy, ns * sizeof(double), cudaMemcpyDeviceToHost, sl.st));
    SN_CUDA(cudaMemcpyAsync(sl.h_virial, sl.virial, ns * 9 * sizeof(double), cudaMemcpyDeviceToHost, sl.st));
    SN_CUDA(cudaMemcpyAsync(sl.h_forces, sl.forces, N * 3 * sizeof(double), cudaMemcpyDeviceToHost, sl.st));
    SN_CUDA(cudaMemcpyAsync(sl.h_flags, sl.ws->flags, FLAG_WORDS * sizeof(int), cudaMemcpyDeviceToHost, sl.st));
    SN_CUDA(cudaEventRecord(sl.ev, sl.st));
    sl.off = b.atom_off;
    sl.batch = std::move(b);
    return SEVENNET_OK;
}

// A batch whose edge list outgrew the slot's capacity runs again, synchronously,
// through eval_batch (which enlarges the workspace); rare by construction.
static sevennet_status slot_rerun(sevennet_server* S, SrvSlot& sl) {
    const int32_t ns = sl.batch.n_structs;
    const int64_t N = sl.batch.atom_off[ns];
    SN_TRY(eval_batch(S->M, sl.ws, sl.batch, sl.species, sl.pos, S->prec, sl.energy, sl.forces, sl.virial, sl.st));
    SN_CUDA(cudaMemcpyAsync(sl.h_energy, sl.energy, ns * sizeof(double), cudaMemcpyDeviceToHost, sl.st));
    SN_CUDA(cudaMemcpyAsync(sl.h_virial, sl.virial, ns * 9 * sizeof(double), cudaMemcpyDeviceToHost, sl.st));
    SN_CUDA(cudaMemcpyAsync(sl.h_forces, sl.forces, N * 3 * sizeof(double), cudaMemcpyDeviceToHost, sl.st));
    SN_CUDA(cudaStreamSynchronize(sl.st));
    return SEVENNET_OK;
}

static void slot_finish(sevennet_server* S, SrvSlot& sl, sevennet_status status) {
    if (status == SEVENNET_OK) {
        if (sl.h_flags[FLAG_EDGE_OVERFLOW]) status = slot_rerun(S, sl);
        else status = check_flags(sl.h_flags);
    }
    const double now = srv_now(S);
    std::lock_guard<std::mutex> lk(S->mu);
    for (size_t i = 0; i < sl.reqs.size(); ++i) {
        SrvRes& r = S->results[sl.reqs[i].ticket];
        r.done = true;
        r.status = status;
        r.submit_s = sl.reqs[i].submit_s;
        r.start_s = sl.start_s;
        r.done_s = now;
        r.batch_id = sl.batch_id;
        r.batch_structs = (int32_t)sl.reqs.size();
        if (status == SEVENNET_OK) {
            r.energy = sl.h_energy[i];
            std::copy(sl.h_virial + i * 9, sl.h_virial + i * 9 + 9, r.virial);
            r.forces.assign(sl.h_forces + sl.off[i] * 3, sl.h_forces + sl.off[i + 1] * 3);
        }
    }
    S->in_flight -= sl.bytes;
    sl.reqs.clear();
    sl.busy = false;
    sl.bytes = 0;
}

static void server_loop(sevennet_server* S) {
    cudaSetDevice(S->M->device);
    while (true) {
        bool progressed = false;
        // 1. retire finished batches
        for (auto& sl : S->slots) {
            if (sl.busy && cudaEventQuery(sl.ev) == cudaSuccess) {
                slot_finish(S, sl, SEVENNET_OK);
                progressed = true;
            }
        }
        // 2. admit queued requests into a free slot
        SrvSlot* free_slot = nullptr;
        for (auto& sl : S->slots) if (!sl.busy) { free_slot = &sl; break; }
        if (free_slot) {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->stop && S->queue.empty()) break;
            size_t bytes = 0;
            int64_t atoms = 0;
            while (!S->queue.empty() && (int32_t)free_slot->reqs.size() < S->max_structs &&
                   atoms + S->queue.front().n <= free_slot->cap_atoms) {
                bytes += S->queue.front().bytes;
                atoms += S->queue.front().n;
                free_slot->reqs.push_back(std::move(S->queue.front()));
                S->queue.pop_front();
            }
            if (!free_slot->reqs.empty()) {
                S->in_flight += bytes;
                free_slot->bytes = bytes;
                free_slot->busy = true;
                free_slot->batch_id = S->next_batch++;
                lk.unlock();
                const sevennet_status st = slot_launch(S, *free_slot);
                if (st != SEVENNET_OK) {
                    cudaStreamSynchronize(free_slot->st);
                    slot_finish(S, *free_slot, st);
                }
                progressed = true;
            }
        } else {
            std::lock_guard<std::mutex> lk(S->mu);
            if (S->stop && S->queue.empty()) {
                bool any = false;
                for (auto& sl : S->slots) any |= sl.busy;
                if (!any) break;
            }
        }
        if (!progressed) {
            std::unique_lock<std::mutex> lk(S->mu);
            bool any_busy = false;
            for (auto& sl : S->slots) any_busy |= sl.busy;
            if (S->stop && S->queue.empty() && !any_busy) break;
            S->cv.wait_for(lk, std::chrono::microseconds(any_busy ? 50 : 500));
        }
    }
}

}  // namespace sn

extern "C" {

sevennet_status sevennet_server_create(sevennet_model* M, size_t hbm_budget_bytes, int32_t n_streams,
                                       int32_t max_batch_structs, sevennet_precision prec, sevennet_server** out) {
    SN_CHECK(M && out && n_streams >= 1 && n_streams <= 16 && max_batch_structs >= 1 && hbm_budget_bytes > 0,
             SEVENNET_EINVAL, "bad argument");
    SN_CHECK(prec == SEVENNET_FP32 || prec == SEVENNET_BF16, SEVENNET_EINVAL, "unknown precision");
    *out = nullptr;
    SN_ENTER(M->device);
    auto* S = new sevennet_server();
    S->M = M;
    S->budget = hbm_budget_bytes;
    S->max_structs = max_batch_structs;
    S->prec = prec;
    S->t0 = std::chrono::steady_clock::now();
    S->slots.resize(n_streams);
    for (auto& sl : S->slots) {
        if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            set_error("server: stream creation failed");
            sevennet_server_destroy(S);
            return SEVENNET_ECUDA;
        }
        sl.ws = new Workspace();
    }
    // each slot owns an equal share of the budget, allocated now
    S->slot_atoms = (int64_t)((hbm_budget_bytes / (size_t)n_streams) / bytes_per_atom(M));
    for (auto& sl : S->slots) {
        const sevennet_status s = slot_alloc(M, sl, S->slot_atoms, max_batch_structs);
        if (s != SEVENNET_OK) {
            sevennet_server_destroy(S);
            return s;
        }
    }
    S->worker = std::thread(server_loop, S);
    *out = S;
    return SEVENNET_OK;
}

sevennet_status sevennet_server_submit(sevennet_server* S, const sevennet_request* req, uint64_t* ticket) {
    SN_CHECK(S && req && ticket && req->n_atoms >= 1 && req->species && req->pos && req->cell, SEVENNET_EINVAL,
             "bad request");
    for (int64_t i = 0; i < req->n_atoms; ++i)
        SN_CHECK(req->species[i] >= 0 && req->species[i] < S->M->cfg.n_species, SEVENNET_EINVAL,
                 "species index out of range");
    for (int64_t i = 0; i < 3 * req->n_atoms; ++i)
        SN_CHECK(std::isfinite(req->pos[i]), SEVENNET_EINVAL, "position not finite");
    SrvReq r;
    r.n = req->n_atoms;
    r.species.assign(req->species, req->species + req->n_atoms);
    r.pos.assign(req->pos, req->pos + 3 * req->n_atoms);
    std::copy(req->cell, req->cell + 9, r.cell);
    r.bytes = predict_bytes(S->M, r.n);
    SN_CHECK(r.n <= S->slot_atoms, SEVENNET_ENOMEM_ADMIT,
             "request of %lld atoms needs %zu bytes; a slot holds %lld atoms (its share of the %zu-byte budget)",
             (long long)r.n, r.bytes, (long long)S->slot_atoms, S->budget);
    r.submit_s = srv_now(S);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r.ticket = S->next_ticket++;
        *ticket = r.ticket;
        S->results[r.ticket] = SrvRes();
        S->queue.push_back(std::move(r));
    }
    S->cv.notify_one();
    return SEVENNET_OK;
}

sevennet_status sevennet_server_poll(sevennet_server* S, uint64_t ticket, sevennet_result* res, int* done) {
    SN_CHECK(S && done, SEVENNET_EINVAL, "bad argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->results.find(ticket);
    SN_CHECK(it != S->results.end(), SEVENNET_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    if (!it->second.done) {
        *done = 0;
        return SEVENNET_OK;
    }
    *done = 1;
    const SrvRes& r = it->second;
    const sevennet_status st = r.status;
    if (res) {
        res->energy = r.energy;
        std::copy(r.virial, r.virial + 9, res->virial);
        if (res->forces) std::copy(r.forces.begin(), r.forces.end(), res->forces);
        res->submit_s = r.submit_s;
        res->start_s = r.start_s;
        res->done_s = r.done_s;
        res->batch_id = r.batch_id;
        res->batch_structs = r.batch_structs;
    }
    S->results.erase(it);
    if (st != SEVENNET_OK) set_error("request failed with status %d", st);
    return st;
}

double sevennet_server_now(const sevennet_server* S) { return S ? srv_now(S) : 0.0; }

void sevennet_server_destroy(sevennet_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->queue.clear();
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    cudaSetDevice(S->M->device);
    for (auto& sl : S->slots) {
        if (sl.st) cudaStreamSynchronize(sl.st);
        cudaFree(sl.pos); cudaFree(sl.forces); cudaFree(sl.species); cudaFree(sl.energy); cudaFree(sl.virial);
        cudaFreeHost(sl.h_pos); cudaFreeHost(sl.h_forces); cudaFreeHost(sl.h_species);
        cudaFreeHost(sl.h_energy); cudaFreeHost(sl.h_virial); cudaFreeHost(sl.h_flags);
        ws_free(sl.ws);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.st) cudaStreamDestroy(sl.st);
    }
    delete S;
}

}  // extern "C"
