/*
 * sevennet.h -- C ABI of the GB300 (sm_103a) SevenNet energy / force / virial library.
 *
 * The library evaluates a NequIP-style equivariant message-passing potential
 * (SevenNet, arXiv:2402.03789) on periodic cells: a cell-list neighbour build,
 * edge featurisation, per-edge radial MLP, Clebsch-Gordan tensor-product
 * convolution with a segmented sum into receivers, gated self-interaction
 * linears, an atomwise readout, and forces / virial as -dE/dr and -dE/d(strain).
 * Every step is a hand-written CUDA kernel; nothing runs on the CPU except
 * argument checks, planning and copies.
 *
 * Conventions shared by all entry points
 *   Units        : positions A, energies eV, forces eV/A, virial eV, masses amu,
 *                  time fs, velocities A/fs.
 *   Cells        : cell[3][3] row-major, rows are the lattice vectors a, b, c.
 *   Positions    : any real values; periodic images are found whatever the
 *                  wrapping of the input.
 *   Ownership    : the caller owns every buffer it passes; inputs are copied,
 *                  outputs are written into caller storage.  Opaque handles are
 *                  owned by the library and freed by the matching *_destroy.
 *   Errors       : functions return 0 on success or a negative status; the
 *                  message of the last failure on the calling thread is
 *                  returned by sevennet_last_error().  No call aborts or traps.
 *   Threads      : one model may be used from one thread at a time, except the
 *                  server API, which is thread-safe.
 *   Precision    : SEVENNET_FP32 computes every step in FP32 (FFMA, no TF32);
 *                  SEVENNET_BF16 runs the radial-MLP and node-linear matrix
 *                  products on tensor cores with BF16 operands and FP32
 *                  accumulation.  Distances and spherical harmonics are FP32;
 *                  per-structure energy and virial sums and the MD update are
 *                  FP64 in both.
 *
 * Model definition (paper Sec. 2 Eqs. 1-4, Figure 2; Sec. 3.2 "identical to
 * NequIP"; Sec. 5.1 SevenNet-0).  With l_max = lmax and mul[l] channels per
 * irrep l (features mul[0]x0e + mul[1]x1e + ...):
 *   h1_v        = W_emb[species_v]                                   (mul[0] scalars)
 *   per block t : sc = LinSC(h), x = Lin1(h),
 *                 w_e = MLP(B(r_e)), B = Bessel_n(r) * envelope(r),
 *                   Bessel_n(r) = (2/r_c) sin(n pi r / r_c) / r, n = 1..n_basis,
 *                   envelope(x=r/r_c) = 1 - (p+1)(p+2)/2 x^p + p(p+2) x^(p+1)
 *                                       - p(p+1)/2 x^(p+2)   (x < 1), 0 otherwise,
 *                   MLP = n_basis -> H -> H -> W with SiLU after the hidden
 *                   layers, no biases, each layer scaled by 1/sqrt(fan_in);
 *                 m_v = 1/avg_num_neigh * sum_{edges e into v} TP(x_src(e), Y(d_e); w_e),
 *                   TP: channel-wise ("uvu") coupling over the paths
 *                   (l1, l2, l3), |l1-l2| <= l3 <= min(l1+l2, lmax), l1 in the
 *                   block input, l2 <= lmax; the last block keeps l3 = 0 only;
 *                 y = Lin2(m) + sc;  h' = Gate(y): SiLU on the mul[0] scalars,
 *                   SiLU(gate) * y_l for l >= 1 (gates ordered l = 1, 2, ...);
 *                   the last block has y = mul[0] scalars and h' = SiLU(y).
 *   E_v = scale * R1(R0(h_v)) + shift[species_v],   E = sum_v E_v     (Eq. 1)
 *   F_v = -dE/dr_v (Eq. 2) = sum_w (F_vw - F_wv), F_vw = dE/dd_vw   (Eqs. 5-7)
 *   W_ab = -dE/d(eps_ab) under r -> (I + eps) r, cell rows likewise
 *        = -sum_edges (dE/dd_e)_a (d_e)_b
 *   Linears act per irrep on the channel index: out = in @ W / sqrt(mul_in).
 *   Spherical harmonics: real, z polar axis, m = -l..l, component normalised
 *   (sum_m Y_lm^2 = 2l+1): Y1 = sqrt3 (y, z, x); Y2 = (sqrt15 xy, sqrt15 yz,
 *   sqrt5/2 (3z^2-1), sqrt15 xz, sqrt15/2 (x^2-y^2)).  Coupling tensors: complex
 *   Clebsch-Gordan coefficients carried to this real basis, the non-zero real or
 *   imaginary part kept, scaled to sum C^2 = 2 l3 + 1, sign fixed so that the
 *   first entry in (m1, m2, m3) order with |C| > 1e-9 is positive.
 *
 * Canonical weight vector (FP64, copied at model creation): embed
 * [n_species][mul0]; per block t: sc[l] [mul_in_l][mul_y_l] for each l present
 * in both h and y (ascending), lin1[l] [mul_in_l][mul_in_l] for l in h,
 * mlp0 [n_basis][H], mlp1 [H][H], mlp2 [H][W] (W columns path-major,
 * channel-minor), lin2[l] [mul_msg_l][mul_y_l] for l with messages; then
 * readout0 [mul0][readout_hidden], readout1 [readout_hidden][1].  Row index =
 * input channel.  sevennet_n_params() returns the length.
 */
#ifndef SEVENNET_H
#define SEVENNET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int sevennet_status;

#define SEVENNET_OK            0
#define SEVENNET_EINVAL       -1   /* bad argument, shape, species index, coincident atoms */
#define SEVENNET_ENOMEM       -2   /* device or host allocation failed */
#define SEVENNET_ECUDA        -3   /* a CUDA call failed; message in sevennet_last_error */
#define SEVENNET_EOVERFLOW    -4   /* a capacity was exceeded and could not be grown */
#define SEVENNET_ETIMEDOUT    -5   /* a bounded wait ran out */
#define SEVENNET_ENOMEM_ADMIT -6   /* serving: request larger than the HBM budget */
#define SEVENNET_EAGAIN       -7   /* serving: result not ready yet */

typedef enum { SEVENNET_FP32 = 0, SEVENNET_BF16 = 1 } sevennet_precision;

typedef struct sevennet_model sevennet_model;     /* opaque, library-owned */
typedef struct sevennet_nlist sevennet_nlist;     /* opaque, device-resident neighbour list */
typedef struct sevennet_md sevennet_md;           /* opaque MD state, device-resident */
typedef struct sevennet_server sevennet_server;   /* opaque serving loop */

/* Model hyper-parameters (Sec. 5.1; lmax 3 for the benchmark models of
 * Sec. 4).  lmax is 1, 2 or 3 (3 needs mlp_hidden 64); every mul[l]
 * (l <= lmax) is a multiple of 32 in [32, 256], entries above lmax are
 * ignored; n_basis <= 16; mlp_hidden is 32 or 64; readout_hidden <= 1024.
 * shift may be NULL (all zero); it is copied. */
typedef struct {
    int32_t n_species;
    int32_t n_layers;
    int32_t lmax;
    int32_t mul[4];
    double  r_cut;
    int32_t n_basis;
    int32_t poly_p;
    int32_t mlp_hidden;
    double  avg_num_neigh;
    int32_t readout_hidden;
    double  scale;
    const double* shift;
} sevennet_model_config;

/* Message of the last failure on this thread (never NULL). */
const char* sevennet_last_error(void);

/* Length of the canonical weight vector for cfg, or -1 if cfg is invalid. */
int64_t sevennet_n_params(const sevennet_model_config* cfg);

/* Build a model on CUDA device `device` from the canonical FP64 weight vector
 * (length n_weights = sevennet_n_params(cfg); copied, converted to FP32 and
 * BF16 device copies).  Paper Sec. 5.1 (hyper-parameters), Figure 2 (blocks).
 * Multiplicities cfg->mul[l] may be any value in [1, 256] (the 4-64 channel
 * models of Sec. 4); those that are not multiples of 32 run as the exact
 * zero-padded model of sevennet_padded_weights (same energy, forces and
 * virial; normalised by the true fan-in). */
/* Host only (no GPU needed): the model the library runs for cfg.  Each
 * multiplicity is rounded up to a multiple of 32 (written to mul_out[4], unused
 * entries 0) and the canonical weights are copied into the padded layout with
 * zeros for the added channels; the linears (self-connection, linear_1,
 * linear_2, readout) are multiplied by sqrt(padded fan-in / true fan-in), so the
 * library's 1/sqrt(fan-in) of the padded model equals the true one.  The added
 * channels stay zero through every operation, so the padded model is exact.
 * out (may be NULL) receives the padded vector, n_out entries (the
 * sevennet_n_params of the padded configuration).  EINVAL for a bad config, a
 * wrong n_weights or a wrong n_out. */
sevennet_status sevennet_padded_weights(const sevennet_model_config* cfg, const double* weights,
                                        size_t n_weights, int32_t* mul_out, double* out, size_t n_out);
sevennet_status sevennet_create_model(const sevennet_model_config* cfg,
                                      const double* weights, size_t n_weights,
                                      int device, sevennet_model** out);
void sevennet_destroy_model(sevennet_model* model);

/* Neighbour list of one cell (Sec. 2: nodes joined when |r_w - r_v| < r_c).
 * Directed edges (v, w, S): receiver v, sender w, integer image S, with
 * d = r_w - r_v + S @ cell, 0 < |d| < r_c; every periodic image counts,
 * self-images (w = v, S != 0) included.  pbc[i] = 0 disables images along
 * lattice vector i.  pos: host [n_atoms][3].  On success *out is a
 * device-resident list and *n_edges its length.  EINVAL for n_atoms < 0, a
 * singular cell or two atoms closer than 1e-8 A. */
sevennet_status sevennet_build_neighbors(sevennet_model* model, int64_t n_atoms,
                                         const double* pos, const double* cell,
                                         const int32_t pbc[3], sevennet_nlist** out,
                                         int64_t* n_edges);
/* Copy a list to host buffers (each [n_edges], shift [n_edges][3]), atom
 * indices in the caller's order, edges in the library's order. */
sevennet_status sevennet_nlist_export(const sevennet_nlist* nl, int32_t* dst,
                                      int32_t* src, int32_t* shift);
void sevennet_nlist_destroy(sevennet_nlist* nl);

/* One energy, force and virial evaluation of one cell from host buffers
 * (Eqs. 1, 2, 5-7; stress virial Sec. 3.2).  species: host [n_atoms] indices
 * into the model's species table; pos host [n_atoms][3]; outputs: energy
 * (1 double), forces host [n_atoms][3], virial host [3][3] (any may be NULL).
 * The call builds the neighbour list, runs every kernel on the model's stream
 * and synchronises before returning. */
sevennet_status sevennet_eval_energy_forces_virial(sevennet_model* model, int64_t n_atoms,
                                                   const int32_t* species, const double* pos,
                                                   const double* cell, const int32_t pbc[3],
                                                   sevennet_precision prec, double* energy,
                                                   double* forces, double* virial);

/* Batched evaluation on device buffers, stream-ordered on `stream`
 * (a cudaStream_t; NULL = the CUDA default stream, as everywhere in CUDA).  n_structs independent
 * periodic cells; structure s owns atoms [atom_offsets[s], atom_offsets[s+1]).
 * Host arrays: atom_offsets [n_structs+1], cells [n_structs][3][3],
 * pbc [n_structs][3] (NULL = all periodic).  Device arrays: species [N],
 * pos [N][3]; outputs energy [n_structs], forces [N][3], virial
 * [n_structs][3][3].  The neighbour build keeps its edge count on the device
 * (edge arrays preallocated at 64 per atom or the largest count seen); the
 * call synchronises once, at its end, to read the status words, and reruns
 * once with more room if the device reported more edges than the capacity.
 * Results are bit-for-bit repeatable; in FP32 a structure's results are the
 * same bits alone and in any batch, in BF16 they agree to BF16 rounding (the
 * tensor-core forward groups a receiver's edges from chunk boundaries that
 * move with the batch). */
sevennet_status sevennet_eval_batch_dev(sevennet_model* model, int32_t n_structs,
                                        const int64_t* atom_offsets, const double* cells,
                                        const int32_t* pbc, const int32_t* species_dev,
                                        const double* pos_dev, sevennet_precision prec,
                                        double* energy_dev, double* forces_dev,
                                        double* virial_dev, void* stream);

/* One message-passing convolution (Eq. 3 with the uvu tensor product of
 * Figure 2b) of block `layer`, on device buffers, for the autograd wrapper.
 *   row_ptr [n_atoms+1], src [n_edges] (int32): edges sorted by receiver;
 *   d [n_edges][3] FP32 displacement r_src - r_recv (+ image);
 *   x [n_atoms][x_dim] FP32 block input after linear_1, irreps stored as
 *     [l][m][channel] blocks; m_out [n_atoms][m_dim] FP32 messages, paths
 *     concatenated per l3 in path order.
 * Backward (the adjoint, Eqs. 5 and 8): given g_m, writes g_x (overwritten) and adds dE/dd into g_d
 * (accumulated; zero it first).  prec selects the arithmetic: FP32 throughout,
 * or BF16 operands with FP32 accumulation for the radial-MLP products and, in
 * the forward, the tensor-product contraction (on tensor cores; x must then be
 * 16-byte aligned, otherwise the FP32-lane contraction runs).  g_x is summed
 * over edges as 64-bit fixed point (order-independent, so the result is
 * repeatable bit for bit); a contribution of magnitude >= 2^16 makes its g_x
 * entry NaN.  Both are ordered on `stream` (NULL = the CUDA default stream)
 * and return without synchronising; their scratch comes from cudaMallocAsync
 * on that stream. */
sevennet_status sevennet_conv_forward_dev(sevennet_model* model, int32_t layer,
                                          int64_t n_atoms, int64_t n_edges,
                                          const int32_t* row_ptr, const int32_t* src,
                                          const float* d, const float* x, float* m_out,
                                          sevennet_precision prec, void* stream);
sevennet_status sevennet_conv_backward_dev(sevennet_model* model, int32_t layer,
                                           int64_t n_atoms, int64_t n_edges,
                                           const int32_t* row_ptr, const int32_t* src,
                                           const float* d, const float* x, const float* g_m,
                                           float* g_x, float* g_d, sevennet_precision prec,
                                           void* stream);
/* The forward of sevennet_conv_forward_dev for callers that may not allocate
 * device memory during the call (a fixed memory plan, or code that must not
 * risk the synchronisation an allocation or free can bring).  No counterpart
 * in the paper.  Arguments, layouts and results are those of
 * sevennet_conv_forward_dev; the per-edge scratch lives in one static device
 * array of the library (5 MiB, held by every GPU that loads the library until
 * exit) instead of being allocated.  Limits and behaviour:
 *   - n_edges <= 262144, else EINVAL and nothing is launched;
 *   - no cudaMalloc / cudaFree / allocating library call is made;
 *   - the first call on a device looks up the array's address (set-up), so
 *     make that first call before any stream capture;
 *   - every call reuses the same array: calls whose kernels overlap on the GPU
 *     race; order them on one stream or with events.
 * row_ptr must be a valid CSR (row_ptr[0] = 0, row_ptr[n_atoms] = n_edges). */
sevennet_status sevennet_conv_forward_noalloc(sevennet_model* model, int32_t layer,
                                              int64_t n_atoms, int64_t n_edges,
                                              const int32_t* row_ptr, const int32_t* src,
                                              const float* d, const float* x, float* m_out,
                                              sevennet_precision prec, void* stream);
/* Row widths used by the conv entry points: x_dim and m_dim of block layer. */
sevennet_status sevennet_conv_dims(const sevennet_model* model, int32_t layer,
                                   int32_t* x_dim, int32_t* m_dim);

/* Single-process emulation of the paper's multi-GPU spatial decomposition
 * (Sec. 3.1, Figure 3) on one GPU: the cell is cut into n_domains slabs along
 * its first lattice vector; each domain evaluates its own atoms with ghost
 * copies of the atoms within r_c of them, exchanging h after every block
 * (forward) and dE/dh and the partial edge forces backwards through device
 * buffers.  Same arguments and outputs as sevennet_eval_energy_forces_virial
 * (all periodic); the result equals the single-domain evaluation up to FP
 * summation order.  A check of the decomposition scheme, not a fast path: it
 * builds the domain graphs on the host.  EINVAL for n_domains outside [1, 64]
 * and as sevennet_eval_energy_forces_virial. */
sevennet_status sevennet_eval_decomposed(sevennet_model* model, int64_t n_atoms,
                                         const int32_t* species, const double* pos,
                                         const double* cell, int32_t n_domains,
                                         sevennet_precision prec, double* energy,
                                         double* forces, double* virial);

/* Molecular dynamics: velocity Verlet in FP64 on the device (NVE by default),
 * neighbour list rebuilt every step unless a skin is set.  masses: amu per
 * species [n_species]; vel A/fs.  Positions, velocities and forces stay on the
 * device between steps.  The paper drives its MD from LAMMPS (Sec. 3.2) with
 * NVT runs in Sec. 4 and a melt-quench in Sec. 5.2. */
sevennet_status sevennet_md_create(sevennet_model* model, int64_t n_atoms,
                                   const int32_t* species, const double* pos,
                                   const double* vel, const double* masses,
                                   const double* cell, sevennet_precision prec,
                                   sevennet_md** out);
/* Advance n_steps steps of dt_fs.  epot_log / ekin_log (host [n_steps] or
 * NULL) receive E_pot and E_kin after each step.  The steps are enqueued
 * without host synchronisation: neighbour lists keep their edge counts on the
 * device, the Verlet-skin rebuild is decided on the device, and the call
 * synchronises once, at the end.  If an edge list outgrew its preallocated
 * capacity (reported by the device), the call restores the state it started
 * from, enlarges the capacity and runs the steps again (a second
 * synchronisation, rare); a second overflow returns EOVERFLOW. */
sevennet_status sevennet_md_step(sevennet_md* md, int64_t n_steps, double dt_fs,
                                 double* epot_log, double* ekin_log);
/* Host copies of the current state (each may be NULL). */
sevennet_status sevennet_md_get_state(const sevennet_md* md, double* pos, double* vel,
                                      double* forces);
/* Verlet list with a skin (A, >= 0; 0 = rebuild every step, the default).
 * With skin > 0 the neighbour list is built for r_c + skin and reused: each
 * step keeps its pairs within r_c at the current positions (same edge set as a
 * full build, in list order), and a new list is built once an atom has moved
 * more than skin / 2 since the last build.  The energy, forces and virial are
 * those of the full build up to FP summation order.  EINVAL for a negative or
 * non-finite skin. */
sevennet_status sevennet_md_set_skin(sevennet_md* md, double skin_A);
/* Nose-Hoover NVT (Sec. 4 runs NVT; the paper gives no thermostat settings):
 * one thermostat, dv/dt = F/m - xi v, dxi/dt = (2 K - N_f k_B T0) / Q,
 * deta/dt = xi, N_f = 3N - 3, Q = N_f k_B T0 tau^2; each step is
 * thermostat(dt/2), velocity Verlet(dt), thermostat(dt/2).  tau_fs <= 0 turns
 * the thermostat off (NVE).  xi and eta persist across calls, so a schedule
 * may set a new temperature between md_step calls.  EINVAL
 * for non-finite arguments, temperature <= 0 with tau > 0, or fewer than two
 * atoms. */
sevennet_status sevennet_md_set_nose_hoover(sevennet_md* md, double temperature_K, double tau_fs);
/* Nose-Hoover NVT whose target ramps linearly from t_start_K to t_end_K over
 * the next n_steps steps (counted across md_step calls), then stays at
 * t_end_K: the melt-quench schedule of Sec. 5.2 (hold at 5000 K, hold at
 * 3000 K, quench at -33 K/ps) is a sequence of holds and ramps.  Step k of the
 * ramp (k = 0 .. n_steps - 1) uses T0 = t_start + (t_end - t_start)(k + 1/2) /
 * n_steps for both thermostat half-steps, and Q = N_f k_B T0 tau^2 follows
 * T0.  xi and eta carry over.  EINVAL for non-finite arguments, tau <= 0,
 * temperatures <= 0, n_steps < 1 or fewer than two atoms. */
sevennet_status sevennet_md_set_nose_hoover_ramp(sevennet_md* md, double t_start_K, double t_end_K,
                                                 int64_t n_steps, double tau_fs);
/* Thermostat state: xi (1/fs) and eta (dimensionless); the conserved extended
 * energy is E_pot + E_kin + Q xi^2 / 2 + N_f k_B T0 eta.  Synchronises. */
sevennet_status sevennet_md_get_nose_hoover(const sevennet_md* md, double* xi, double* eta);
/* Neighbour-list builds so far (the initial evaluation counts as one) and the
 * edge count of the last refreshed Verlet list (0 without a skin). */
sevennet_status sevennet_md_get_stats(const sevennet_md* md, int64_t* n_builds, int64_t* n_edges);
void sevennet_md_destroy(sevennet_md* md);

/* Serving: continuous batching of independent structures.  Requests are
 * copied at submission.  At creation the HBM budget is split evenly over
 * n_streams slots and each slot's workspace and pinned buffers are allocated
 * for the atoms its share holds (about 47 KB per atom for SevenNet-0), so
 * running a batch allocates and frees nothing and waits for nothing on the
 * host.  A worker thread packs queued requests into a free slot (up to
 * max_batch_structs structures and the slot's atoms), enqueues copy-in,
 * neighbour build, evaluation and copy-out on the slot's stream, and retires
 * batches by event; batches overlap on the GPU and new arrivals join the next
 * batch without waiting for the running ones.  The results of a structure do
 * not depend on the batch it ran in beyond FP summation order (bit-identical in
 * FP32). */
typedef struct {
    int64_t        n_atoms;
    const int32_t* species;   /* host [n_atoms] */
    const double*  pos;       /* host [n_atoms][3] */
    const double*  cell;      /* host [3][3] */
} sevennet_request;

typedef struct {
    double  energy;           /* eV */
    double* forces;           /* caller buffer [n_atoms][3], filled by poll */
    double  virial[9];        /* eV */
    double  submit_s;         /* seconds on the server clock */
    double  start_s;          /* when its batch was launched */
    double  done_s;
    int32_t batch_id;         /* batch the request ran in */
    int32_t batch_structs;    /* structures in that batch */
} sevennet_result;

sevennet_status sevennet_server_create(sevennet_model* model, size_t hbm_budget_bytes,
                                       int32_t n_streams, int32_t max_batch_structs,
                                       sevennet_precision prec, sevennet_server** out);
/* Queue a request; *ticket identifies it.  ENOMEM_ADMIT if it has more atoms
 * than one slot holds (it could never run). */
sevennet_status sevennet_server_submit(sevennet_server* s, const sevennet_request* req,
                                       uint64_t* ticket);
/* Non-blocking: *done = 1 and the result copied (forces into res->forces) once
 * the request finished, else *done = 0.  A finished ticket is released by a
 * successful poll. */
sevennet_status sevennet_server_poll(sevennet_server* s, uint64_t ticket,
                                     sevennet_result* res, int* done);
/* Seconds on the server clock (the clock of submit_s / done_s). */
double sevennet_server_now(const sevennet_server* s);
void sevennet_server_destroy(sevennet_server* s);

/* Diagnostics (no counterpart in the paper; used for measurement).
 * sevennet_profile(model, 1) makes every later evaluation on that model record
 * CUDA events around each kernel family on the stream it runs on
 * ("neighbors", "linear", "conv_fwd", "conv_bwd", "gate", "other");
 * sevennet_profile_read() synchronises, adds the recorded intervals up and
 * returns, per family, the total milliseconds and launches (names: n_max
 * entries of 32 chars).  Enabling again clears the totals.
 * sevennet_launch_count() is the number of kernels this library has launched
 * in the process. */
sevennet_status sevennet_profile(sevennet_model* model, int32_t enable);
sevennet_status sevennet_profile_read(sevennet_model* model, int32_t n_max, char* names,
                                      double* total_ms, int64_t* launches, int32_t* n_out);
int64_t sevennet_launch_count(void);

/* FP32 ALU throughput of `device`, measured: a grid of 4 CTAs x 256 threads per
 * SM, each thread updating 16 independent register-resident FMA chains `iters`
 * times (packed = 0: fma.rn.f32; packed = 1: fma.rn.f32x2, two FMAs per
 * instruction).  One untimed warm-up launch, then one launch timed with CUDA
 * events on a private stream.  Writes the FLOPs of the timed launch (2 per FMA)
 * and its milliseconds.  It is the denominator of the ALU roofline of the
 * FP32 path and of the tensor-product phases (the paper gives no kernel-level
 * figure; this is a property of the device).  Allocates and frees one small
 * device buffer; EINVAL for null outputs or iters <= 0, ECUDA on a CUDA error. */
sevennet_status sevennet_fp32_peak(int32_t device, int32_t packed, int32_t iters, double* flop, double* ms);

#ifdef __cplusplus
}
#endif

#endif /* SEVENNET_H */
