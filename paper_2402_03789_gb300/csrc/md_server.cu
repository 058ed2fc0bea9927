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
    unsigned long long* dmax_host = nullptr;
    bool have_list = false;
    // Nose-Hoover thermostat (tau > 0): {xi, eta} on the device
    double nh_T0 = 0.0, nh_tau = 0.0;
    // linear ramp of the target from nh_T0 to nh_T1 over nh_ramp steps (0: none);
    // nh_done steps of it have run
    double nh_T1 = 0.0;
    int64_t nh_ramp = 0, nh_done = 0;
    double* nh = nullptr;
    int64_t n_builds = 0, n_edges = 0;
};

// Forces at the current positions.  Without a skin: a full neighbour build and
// evaluation.  With a skin: the stored Verlet list (cutoff r_c + skin) is rebuilt
// when some atom has moved more than skin / 2 since its build, and otherwise
// filtered to r < r_c at the current positions (no pair can have entered r_c).
static sevennet_status md_evaluate(sevennet_md* md) {
    sevennet_model* M = md->M;
    if (md->skin <= 0.0) {
        SN_TRY(eval_batch(M, md->ws, md->b, md->species, md->pos, md->prec, md->ev, md->f, md->ev + 1, md->st));
        ++md->n_builds;
        return SEVENNET_OK;
    }
    bool rebuild = !md->have_list;
    if (!rebuild) {
        SN_CUDA(cudaMemsetAsync(md->dmax, 0, sizeof(unsigned long long), md->st));
        max_disp_kernel<<<(unsigned)((md->N + 255) / 256), 256, 0, md->st>>>(md->N, md->pos, md->ref, md->dmax);
        SN_CUDA(cudaMemcpyAsync(md->dmax_host, md->dmax, sizeof(unsigned long long), cudaMemcpyDeviceToHost, md->st));
        SN_CUDA(cudaStreamSynchronize(md->st));
        double d2;
        std::memcpy(&d2, md->dmax_host, sizeof(double));
        rebuild = !(d2 <= 0.25 * md->skin * md->skin);
    }
    const int64_t N = md->N;
    if (rebuild) {
        int64_t EL = 0;
        SN_TRY(build_neighbors(M, md->ws, md->b, md->pos, md->species, md->st, &EL, M->cfg.r_cut + md->skin));
        if (EL > md->l_cap) {
            cudaFree(md->l_src);
            cudaFree(md->l_shift);
            md->l_src = md->l_shift = nullptr;
            md->l_cap = 0;
            const int64_t cap = EL + EL / 4 + 1024;
            if (cudaMalloc(&md->l_src, cap * sizeof(int)) || cudaMalloc(&md->l_shift, cap * 3 * sizeof(int))) {
                cudaGetLastError();
                set_error("cudaMalloc failed for the Verlet list");
                return SEVENNET_ENOMEM;
            }
            md->l_cap = cap;
        }
        if (!md->l_row && cudaMalloc(&md->l_row, (N + 1) * sizeof(int))) {
            cudaGetLastError();
            set_error("cudaMalloc failed for the Verlet list");
            return SEVENNET_ENOMEM;
        }
        SN_CUDA(cudaMemcpyAsync(md->l_row, md->ws->row_ptr, (N + 1) * sizeof(int), cudaMemcpyDeviceToDevice, md->st));
        if (EL > 0) {
            SN_CUDA(cudaMemcpyAsync(md->l_src, md->ws->src, EL * sizeof(int), cudaMemcpyDeviceToDevice, md->st));
            SN_CUDA(cudaMemcpyAsync(md->l_shift, md->ws->shift, EL * 3 * sizeof(int), cudaMemcpyDeviceToDevice,
                                    md->st));
        }
        SN_CUDA(cudaMemcpyAsync(md->ref, md->pos, N * 3 * sizeof(double), cudaMemcpyDeviceToDevice, md->st));
        md->have_list = true;
        ++md->n_builds;
    }
    int64_t E = 0;
    SN_TRY(refresh_neighbors(M, md->ws, N, md->pos, md->l_row, md->l_src, md->l_shift, md->st, &E));
    md->n_edges = E;
    SN_TRY(run_model(M, md->ws, md->b, E, md->prec, md->ev, md->f, md->ev + 1, md->st));
    SN_CUDA(cudaMemcpyAsync(md->ws->flags_host, md->ws->flags, 8 * sizeof(int), cudaMemcpyDeviceToHost, md->st));
    SN_CUDA(cudaStreamSynchronize(md->st));
    SN_CHECK(md->ws->flags_host[2] == 0, SEVENNET_ECUDA, "internal error: reverse edge not found");
    return SEVENNET_OK;
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
    if (md->dmax_host) cudaFreeHost(md->dmax_host);
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
        cudaMallocHost(&md->dmax_host, sizeof(unsigned long long))) {
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
    if (cudaMemset(md->nh, 0, 2 * sizeof(double))) {
        set_error("cudaMemset failed");
        return fail(SEVENNET_ECUDA);
    }
    sevennet_status s = eval_batch(M, md->ws, md->b, md->species, md->pos, prec, md->ev, md->f, md->ev + 1, md->st);
    if (s) return fail(s);
    md->n_builds = 1;
    *out = md;
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
    const int64_t n3 = md->N * 3;
    const unsigned blocks = (unsigned)((n3 + 255) / 256);
    const bool nvt = md->nh_tau > 0.0;
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
    if (n_steps > 0) {
        if (epot_log) SN_CUDA(cudaMemcpyAsync(epot_log, md->epot, n_steps * sizeof(double), cudaMemcpyDeviceToHost, md->st));
        if (ekin_log) SN_CUDA(cudaMemcpyAsync(ekin_log, md->ekin, n_steps * sizeof(double), cudaMemcpyDeviceToHost, md->st));
    }
    SN_CUDA(cudaStreamSynchronize(md->st));
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
    std::chrono::steady_clock::time_point t0;
};

namespace sn {

static double srv_now(const sevennet_server* s) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

// Predicted device bytes of one request: activations per atom plus per-edge
// arrays at a generous 80 neighbours per atom.
static size_t predict_bytes(const sevennet_model* M, int64_t n) {
    const size_t per_atom = (size_t)(M->T * (M->x_max + M->y_max) + M->m_max + M->y_max + M->x_max +
                                     2 * M->h_max) * sizeof(float) + 200;
    const size_t per_edge = 4 * 4 + 12 + 16 + 12;
    return per_atom * (size_t)n + per_edge * (size_t)n * 80 + 4096;
}

static sevennet_status slot_reserve(SrvSlot& sl, int64_t atoms, int32_t structs) {
    if (atoms > sl.cap_atoms) {
        cudaFree(sl.pos); cudaFree(sl.forces); cudaFree(sl.species);
        cudaFreeHost(sl.h_pos); cudaFreeHost(sl.h_forces); cudaFreeHost(sl.h_species);
        const int64_t A = std::max<int64_t>(atoms * 5 / 4, 256);
        if (cudaMalloc(&sl.pos, A * 3 * sizeof(double)) || cudaMalloc(&sl.forces, A * 3 * sizeof(double)) ||
            cudaMalloc(&sl.species, A * sizeof(int32_t)) || cudaMallocHost(&sl.h_pos, A * 3 * sizeof(double)) ||
            cudaMallocHost(&sl.h_forces, A * 3 * sizeof(double)) || cudaMallocHost(&sl.h_species, A * sizeof(int32_t))) {
            cudaGetLastError();
            sl.cap_atoms = 0;
            set_error("server: allocation failed");
            return SEVENNET_ENOMEM;
        }
        sl.cap_atoms = A;
    }
    if (structs > sl.cap_structs) {
        cudaFree(sl.energy); cudaFree(sl.virial); cudaFreeHost(sl.h_energy); cudaFreeHost(sl.h_virial);
        const int32_t S = std::max<int32_t>(structs, 64);
        if (cudaMalloc(&sl.energy, S * sizeof(double)) || cudaMalloc(&sl.virial, S * 9 * sizeof(double)) ||
            cudaMallocHost(&sl.h_energy, S * sizeof(double)) || cudaMallocHost(&sl.h_virial, S * 9 * sizeof(double))) {
            cudaGetLastError();
            sl.cap_structs = 0;
            set_error("server: allocation failed");
            return SEVENNET_ENOMEM;
        }
        sl.cap_structs = S;
    }
    return SEVENNET_OK;
}

// Enqueue one packed batch on a slot (returns after the neighbour count read).
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
    SN_TRY(slot_reserve(sl, N, ns));
    for (int32_t i = 0; i < ns; ++i) {
        std::copy(sl.reqs[i].pos.begin(), sl.reqs[i].pos.end(), sl.h_pos + b.atom_off[i] * 3);
        std::copy(sl.reqs[i].species.begin(), sl.reqs[i].species.end(), sl.h_species + b.atom_off[i]);
    }
    SN_CUDA(cudaMemcpyAsync(sl.pos, sl.h_pos, N * 3 * sizeof(double), cudaMemcpyHostToDevice, sl.st));
    SN_CUDA(cudaMemcpyAsync(sl.species, sl.h_species, N * sizeof(int32_t), cudaMemcpyHostToDevice, sl.st));
    int64_t E = 0;
    SN_TRY(check_batch(b));
    SN_TRY(build_neighbors(S->M, sl.ws, b, sl.pos, sl.species, sl.st, &E));
    SN_TRY(run_model(S->M, sl.ws, b, E, S->prec, sl.energy, sl.forces, sl.virial, sl.st));
    SN_CUDA(cudaMemcpyAsync(sl.h_energy, sl.energy, ns * sizeof(double), cudaMemcpyDeviceToHost, sl.st));
    SN_CUDA(cudaMemcpyAsync(sl.h_virial, sl.virial, ns * 9 * sizeof(double), cudaMemcpyDeviceToHost, sl.st));
    SN_CUDA(cudaMemcpyAsync(sl.h_forces, sl.forces, N * 3 * sizeof(double), cudaMemcpyDeviceToHost, sl.st));
    SN_CUDA(cudaEventRecord(sl.ev, sl.st));
    sl.off = b.atom_off;
    return SEVENNET_OK;
}

static void slot_finish(sevennet_server* S, SrvSlot& sl, sevennet_status status) {
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
            while (!S->queue.empty() && (int32_t)free_slot->reqs.size() < S->max_structs &&
                   S->in_flight + bytes + S->queue.front().bytes <= S->budget) {
                bytes += S->queue.front().bytes;
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
    SN_CHECK(r.bytes <= S->budget, SEVENNET_ENOMEM_ADMIT, "request needs %zu bytes, budget is %zu", r.bytes,
             S->budget);
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
        cudaFreeHost(sl.h_energy); cudaFreeHost(sl.h_virial);
        ws_free(sl.ws);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.st) cudaStreamDestroy(sl.st);
    }
    delete S;
}

}  // extern "C"
