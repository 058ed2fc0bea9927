// C ABI, model construction and the evaluation schedule.
//
// One evaluation (paper Figure 2a: forward path blue, reverse path orange):
//   neighbour build -> embedding -> per block [linear_1 + self-connection,
//   convolution, linear_2, gate] -> readout and FP64 energy -> reverse:
//   per block from the last [gate adjoint, linear_2^T, convolution adjoint
//   (edge gradients dE/dd accumulated over blocks, Eq. 5), linear_1^T and
//   self-connection^T] -> F_v = sum_w (F_vw - F_wv) (Eq. 6) and the virial.
#include "internal.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <atomic>
#include <mutex>

namespace sn {

thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

int num_sms(int device) {
    static int cached[64] = {0};
    if (device < 0 || device >= 64) return 132;
    if (!cached[device]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v <= 0) v = 132;
        cached[device] = v;
    }
    return cached[device];
}

// ---------------------------------------------------------------- convolution set-up
sevennet_status conv_configure_fwd(int H, size_t need);
sevennet_status conv_configure_bwd(int H, size_t need);
sevennet_status conv_configure_bwd_pair(int H, size_t need);
size_t conv_smem_bytes(const ConvDesc& D, int H, bool bwd);

sevennet_status conv_configure(int H, const std::vector<LayerDev>& layers) {
    size_t need_f = 0, need_b = 0, need_tc = 0;
    for (const LayerDev& L : layers) {
        need_f = std::max(need_f, conv_smem_bytes(L.conv, H, false));
        need_b = std::max(need_b, conv_smem_bytes(L.conv, H, true));
        if (L.conv.tc_ok) need_tc = std::max(need_tc, conv_tc_smem_bytes(L.conv, H));
    }
    SN_TRY(conv_configure_fwd(H, need_f));
    SN_TRY(conv_configure_bwd(H, need_b));
    SN_TRY(conv_configure_bwd_pair(H, need_b));
    if (need_tc) SN_TRY(conv_configure_fwd_tc(H, need_tc));
    return SEVENNET_OK;
}

// ---------------------------------------------------------------- diagnostics
static std::atomic<int64_t> g_launch_count{0};

void count_launches(int n) { g_launch_count += n; }

cudaEvent_t Profiler::get() {
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void prof_begin(Profiler* p, int fam, cudaStream_t st, cudaEvent_t* a) {
    (void)fam;
    *a = nullptr;
    if (!p || !p->on) return;
    *a = p->get();
    cudaEventRecord(*a, st);
}

void prof_end(Profiler* p, int fam, cudaStream_t st, cudaEvent_t a, int n_launches) {
    if (!p || !p->on || !a) return;
    cudaEvent_t b = p->get();
    cudaEventRecord(b, st);
    p->pending.push_back({fam, a, b});
    p->launches[fam] += n_launches;
}

// ---------------------------------------------------------------- layer specs
struct PathH { int l1, l2, l3, mul; };

static bool config_valid(const sevennet_model_config* c, std::string* why) {
    auto fail = [&](const char* m) { if (why) *why = m; return false; };
    if (!c) return fail("config is NULL");
    if (c->n_species < 1) return fail("n_species must be >= 1");
    if (c->n_layers < 1 || c->n_layers > 16) return fail("n_layers must be in [1, 16]");
    if (c->lmax < 1 || c->lmax > MAX_LMAX) return fail("lmax must be 1, 2 or 3");
    if (c->lmax == 3 && c->mlp_hidden != 64) return fail("lmax 3 models need mlp_hidden 64");
    for (int l = 0; l <= c->lmax; ++l)
        if (c->mul[l] < 1 || c->mul[l] > 256) return fail("mul[l] must be in [1, 256]");
    if (!(c->r_cut > 0) || !std::isfinite(c->r_cut)) return fail("r_cut must be positive");
    if (c->n_basis < 1 || c->n_basis > MAX_NB) return fail("n_basis must be in [1, 16]");
    if (c->poly_p < 1 || c->poly_p > 32) return fail("poly_p must be in [1, 32]");
    if (c->mlp_hidden != 32 && c->mlp_hidden != 64) return fail("mlp_hidden must be 32 or 64");
    if (!(c->avg_num_neigh > 0)) return fail("avg_num_neigh must be positive");
    if (c->readout_hidden < 1 || c->readout_hidden > 1024) return fail("readout_hidden out of range");
    return true;
}

static void block_irreps(const sevennet_model_config* c, int t, int in_mul[NL], int y_mul[NL],
                         int out_mul[NL], std::vector<PathH>& paths, int msg_mul[NL], bool* last) {
    const int T = c->n_layers, lmax = c->lmax;
    *last = (t == T - 1);
    for (int l = 0; l < NL; ++l) in_mul[l] = y_mul[l] = out_mul[l] = msg_mul[l] = 0;
    if (t == 0) in_mul[0] = c->mul[0];
    else for (int l = 0; l <= lmax; ++l) in_mul[l] = c->mul[l];
    paths.clear();
    for (int l1 = 0; l1 <= MAX_LMAX; ++l1) {
        if (!in_mul[l1]) continue;
        for (int l2 = 0; l2 <= lmax; ++l2)
            for (int l3 = std::abs(l1 - l2); l3 <= std::min(l1 + l2, lmax); ++l3) {
                if (*last && l3 != 0) continue;
                paths.push_back({l1, l2, l3, in_mul[l1]});
                msg_mul[l3] += in_mul[l1];
            }
    }
    if (*last) {
        y_mul[0] = c->mul[0];
        out_mul[0] = c->mul[0];
    } else {
        y_mul[0] = c->mul[0];
        for (int l = 1; l <= lmax; ++l) { y_mul[0] += c->mul[l]; y_mul[l] = c->mul[l]; out_mul[l] = c->mul[l]; }
        out_mul[0] = c->mul[0];
    }
}

static void offsets(const int mul[NL], int off[NL], int* dim) {
    int o = 0;
    for (int l = 0; l < NL; ++l) { off[l] = o; o += (2 * l + 1) * mul[l]; }
    *dim = o;
}

struct WEntry { std::string name; int rows, cols; int64_t off; };

static std::vector<WEntry> weight_entries(const sevennet_model_config* c) {
    std::vector<WEntry> e;
    int64_t off = 0;
    auto add = [&](const std::string& n, int r, int k) { e.push_back({n, r, k, off}); off += (int64_t)r * k; };
    add("embed", c->n_species, c->mul[0]);
    const int H = c->mlp_hidden;
    for (int t = 0; t < c->n_layers; ++t) {
        int in_mul[NL], y_mul[NL], out_mul[NL], msg_mul[NL];
        std::vector<PathH> paths;
        bool last;
        block_irreps(c, t, in_mul, y_mul, out_mul, paths, msg_mul, &last);
        const std::string p = "L" + std::to_string(t) + ".";
        for (int l = 0; l < NL; ++l)
            if (y_mul[l] && in_mul[l]) add(p + "sc." + std::to_string(l), in_mul[l], y_mul[l]);
        for (int l = 0; l < NL; ++l)
            if (in_mul[l]) add(p + "lin1." + std::to_string(l), in_mul[l], in_mul[l]);
        int W = 0;
        for (auto& q : paths) W += q.mul;
        add(p + "mlp0", c->n_basis, H);
        add(p + "mlp1", H, H);
        add(p + "mlp2", H, W);
        for (int l = 0; l < NL; ++l)
            if (y_mul[l] && msg_mul[l]) add(p + "lin2." + std::to_string(l), msg_mul[l], y_mul[l]);
    }
    add("readout0", c->mul[0], c->readout_hidden);
    add("readout1", c->readout_hidden, 1);
    return e;
}

// ---------------------------------------------------------------- small multiplicities
// The kernels give a warp 32 channels of an irrep, so a model whose multiplicity
// of some irrep is not a multiple of 32 (the 4-16 channel models of Sec. 4) runs
// as the model with every multiplicity rounded up to a multiple of 32 and the
// added channels' weights zero.  A zero channel stays zero through every
// operation (linear rows and columns, radial-MLP output columns, SiLU(0) = 0
// gates, readout rows), so energy, forces and virial are those of the original
// model.  The linears are normalised by the true fan-in: the library scales by
// 1/sqrt(padded fan-in), so the copied weights are multiplied by
// sqrt(padded fan-in / true fan-in).
static int pad32(int m) { return (m + 31) / 32 * 32; }

struct PadEntry {
    std::vector<int> rs, cs;    // true row / column segments (each padded separately)
    bool map_rows, map_cols;    // false: identity (sizes that are not multiplicities)
    bool fan_rows;              // normalised by 1/sqrt(rows)
};

static std::vector<PadEntry> pad_entries(const sevennet_model_config* c) {
    std::vector<PadEntry> e;
    const int H = c->mlp_hidden;
    e.push_back({{c->n_species}, {c->mul[0]}, false, true, false});                 // embed
    for (int t = 0; t < c->n_layers; ++t) {
        int in_mul[NL], y_mul[NL], out_mul[NL], msg_mul[NL];
        std::vector<PathH> paths;
        bool last;
        block_irreps(c, t, in_mul, y_mul, out_mul, paths, msg_mul, &last);
        auto yseg = [&](int l) {
            std::vector<int> v;
            if (l == 0 && !last) for (int k = 0; k <= c->lmax; ++k) v.push_back(c->mul[k]);   // scalars, gates
            else v.push_back(y_mul[l]);
            return v;
        };
        for (int l = 0; l < NL; ++l)
            if (y_mul[l] && in_mul[l]) e.push_back({{in_mul[l]}, yseg(l), true, true, true});      // sc
        for (int l = 0; l < NL; ++l)
            if (in_mul[l]) e.push_back({{in_mul[l]}, {in_mul[l]}, true, true, true});            // lin1
        std::vector<int> wseg;
        for (auto& q : paths) wseg.push_back(q.mul);
        e.push_back({{c->n_basis}, {H}, false, false, false});                                   // mlp0
        e.push_back({{H}, {H}, false, false, false});                                            // mlp1
        e.push_back({{H}, wseg, false, true, false});                                            // mlp2
        for (int l = 0; l < NL; ++l)
            if (y_mul[l] && msg_mul[l]) {
                std::vector<int> mseg;
                for (auto& q : paths) if (q.l3 == l) mseg.push_back(q.mul);
                e.push_back({mseg, yseg(l), true, true, true});                                  // lin2
            }
    }
    e.push_back({{c->mul[0]}, {c->readout_hidden}, true, false, true});                         // readout0
    e.push_back({{c->readout_hidden}, {1}, false, false, false});                               // readout1
    return e;
}

static std::vector<int64_t> pad_index(const std::vector<int>& segs, bool map) {
    std::vector<int64_t> idx;
    int64_t base = 0;
    for (int s : segs) {
        for (int i = 0; i < s; ++i) idx.push_back(base + i);
        base += map ? pad32(s) : s;
    }
    return idx;
}

// The padded configuration and its canonical weight vector.
static void pad_model(const sevennet_model_config* c, sevennet_model_config* pc, const double* w,
                      std::vector<double>* wp) {
    *pc = *c;
    for (int l = 0; l <= c->lmax; ++l) pc->mul[l] = pad32(c->mul[l]);
    const auto et = pad_entries(c), ep = pad_entries(pc);
    size_t np = 0;
    for (const auto& e : ep) {
        int64_t R = 0, C = 0;
        for (int r : e.rs) R += r;
        for (int k : e.cs) C += k;
        np += (size_t)(R * C);
    }
    wp->assign(np, 0.0);
    int64_t ot = 0, op = 0;
    for (size_t k = 0; k < et.size(); ++k) {
        const auto ri = pad_index(et[k].rs, et[k].map_rows), ci = pad_index(et[k].cs, et[k].map_cols);
        int64_t Rp = 0, Cp = 0;
        for (int r : ep[k].rs) Rp += r;
        for (int x : ep[k].cs) Cp += x;
        const double sc = et[k].fan_rows ? std::sqrt((double)Rp / (double)ri.size()) : 1.0;
        for (size_t i = 0; i < ri.size(); ++i)
            for (size_t j = 0; j < ci.size(); ++j)
                (*wp)[op + ri[i] * Cp + ci[j]] = w[ot + (int64_t)i * (int64_t)ci.size() + (int64_t)j] * sc;
        ot += (int64_t)ri.size() * (int64_t)ci.size();
        op += Rp * Cp;
    }
}

// ---------------------------------------------------------------- device upload
template <typename T>
static sevennet_status dev_upload(sevennet_model* M, const std::vector<T>& h, T** out) {
    *out = nullptr;
    if (h.empty()) return SEVENNET_OK;
    void* p = nullptr;
    if (cudaMalloc(&p, h.size() * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc of %zu bytes failed", h.size() * sizeof(T));
        return SEVENNET_ENOMEM;
    }
    M->allocations.push_back(p);
    SN_CUDA(cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    *out = static_cast<T*>(p);
    return SEVENNET_OK;
}

static std::vector<float> scaled(const double* w, int rows, int cols, double s, bool transpose) {
    std::vector<float> o((size_t)rows * cols);
    for (int i = 0; i < rows; ++i)
        for (int j = 0; j < cols; ++j) {
            const float v = (float)(w[(size_t)i * cols + j] * s);
            if (transpose) o[(size_t)j * rows + i] = v; else o[(size_t)i * cols + j] = v;
        }
    return o;
}

static std::vector<__nv_bfloat16> to_bf16(const std::vector<float>& f) {
    std::vector<__nv_bfloat16> o(f.size());
    for (size_t i = 0; i < f.size(); ++i) o[i] = __float2bfloat16_rn(f[i]);
    return o;
}

// hi = bf16(w) followed by lo = bf16(w - hi): two BF16 terms that carry w to
// about 16 mantissa bits (used where a tensor-core product takes both).
static std::vector<__nv_bfloat16> to_bf16_pair(const std::vector<float>& f) {
    std::vector<__nv_bfloat16> o(2 * f.size());
    for (size_t i = 0; i < f.size(); ++i) {
        const __nv_bfloat16 h = __float2bfloat16_rn(f[i]);
        o[i] = h;
        o[f.size() + i] = __float2bfloat16_rn(f[i] - __bfloat162float(h));
    }
    return o;
}

static sevennet_status upload_linear(sevennet_model* M, const double* w, int rows, int cols, double s,
                                     float** W, float** WT, __nv_bfloat16** Wh, __nv_bfloat16** WTh) {
    auto a = scaled(w, rows, cols, s, false);
    auto b = scaled(w, rows, cols, s, true);
    SN_TRY(dev_upload(M, a, W));
    SN_TRY(dev_upload(M, b, WT));
    SN_TRY(dev_upload(M, to_bf16_pair(b), Wh));   // [cols][rows] hi, then lo: B operand of out = in @ W
    SN_TRY(dev_upload(M, to_bf16_pair(a), WTh));  // [rows][cols] hi, then lo: B operand of gin = gout @ W^T
    return SEVENNET_OK;
}

// Forward work slots: one path set of input irrep l1 (fwd_path_sets) and a block
// of 32 * CPL channels.  CPL is chosen per set among the compiled widths by
// trying every combination and keeping the one whose longest-first assignment
// to the warps has the smallest maximum load (a slot's load: its multiply-adds
// per edge plus the per-edge gathers and shared-memory loads).  Encoding:
// (l1 << 11) | (set << 8) | (channel block << 2) | log2 CPL.
static bool assign_slots(ConvDesc& D, int H) {
    struct Set { int l1, j, mul, cost, nacc, nG, np; std::vector<int> lcs; };
    std::vector<Set> sets;
    for (int l1 = 0; l1 <= D.lmax; ++l1) {
        if (D.pend[l1] <= D.pbeg[l1]) continue;
        const PathSets S = fwd_path_sets(l1, D.lmax, D.kind);
        const PathList pl = path_list(l1, D.lmax, D.kind);
        for (int j = 0; j < S.n; ++j) {
            Set st{l1, j, D.mul_in[l1], fwd_set_cost(l1, D.lmax, D.kind, j), fwd_set_nacc(l1, D.lmax, D.kind, j), 0,
                   S.b[j + 1] - S.b[j], {}};
            for (int i = S.b[j]; i < S.b[j + 1]; ++i) st.nG += ((2 * l1 + 1) * (2 * pl.l3[i] + 1) + 3) / 4;
            for (int lc = 0; lc < 3; ++lc)
                if (fwd_cpl_compiled(H, l1, st.nacc, 1 << lc) && st.mul % (32 << lc) == 0) st.lcs.push_back(lc);
            if (st.lcs.empty() || st.mul % 32 != 0) return false;
            sets.push_back(st);
        }
    }
    struct Slot { int code, load; };
    auto build = [&](const std::vector<int>& choice, std::vector<Slot>& out) {
        out.clear();
        for (size_t k = 0; k < sets.size(); ++k) {
            const Set& st = sets[k];
            const int lc = st.lcs[choice[k]], cpl = 1 << lc;
            // per edge: multiply-adds, gathers, G quads, weights, edge bookkeeping
            const int load = cpl * st.cost + cpl * (2 * st.l1 + 1) + st.nG + cpl * st.np + 6;
            for (int ub = 0; ub < st.mul / (32 * cpl); ++ub)
                out.push_back({(st.l1 << 11) | (st.j << 8) | (ub << 2) | lc, load});
        }
    };
    auto lpt = [&](std::vector<Slot> sl, int16_t (*grp)[MAX_SLOTS], int16_t* n) {
        std::stable_sort(sl.begin(), sl.end(), [](const Slot& a, const Slot& b) { return a.load > b.load; });
        int load[CONV_WARPS] = {0}, cnt[CONV_WARPS] = {0};
        for (const Slot& x : sl) {
            int best = -1;
            for (int w = 0; w < CONV_WARPS; ++w)
                if (cnt[w] < MAX_SLOTS && (best < 0 || load[w] < load[best])) best = w;
            if (best < 0) return -1;
            if (grp) grp[best][cnt[best]] = (int16_t)x.code;
            ++cnt[best];
            load[best] += x.load;
        }
        if (n) for (int w = 0; w < CONV_WARPS; ++w) n[w] = (int16_t)cnt[w];
        int mx = 0;
        for (int w = 0; w < CONV_WARPS; ++w) mx = std::max(mx, load[w]);
        return mx;
    };
    std::vector<int> choice(sets.size(), 0), best_choice;
    int best = -1;
    std::vector<Slot> sl;
    for (;;) {
        build(choice, sl);
        const int mk = lpt(sl, nullptr, nullptr);
        if (mk >= 0 && (best < 0 || mk < best)) { best = mk; best_choice = choice; }
        size_t k = 0;
        while (k < sets.size() && ++choice[k] == (int)sets[k].lcs.size()) choice[k++] = 0;
        if (k == sets.size()) break;
    }
    if (best < 0) return false;
    build(best_choice, sl);
    return lpt(sl, D.slot_group, D.n_slots) >= 0;
}

// Tensor-core forward tables: B-fragment offsets per path, the staged x
// regions (row strides chosen so that the lanes of a warp read distinct
// shared-memory banks) and the work units (one path set over 16 channels),
// assigned longest-first to the warps.  Blocks with lmax 3, multiplicities not
// divisible by 16 or more shared memory than two CTAs per SM allow keep the
// FFMA forward (tc_ok = 0).
static void assign_tc(ConvDesc& D, int H) {
    D.tc_ok = 0;
    if (D.lmax > 2 || D.x_dim > 4 * 32 * 6) return;     // x rows staged as at most 6 pieces of 16 bytes per lane
    int words = 0, xo = 0;
    for (int l = 0; l < NL; ++l) { D.xs_off[l] = 0; D.xs_stride[l] = 0; }
    for (int l1 = 0; l1 <= D.lmax; ++l1) {
        if (!D.mul_in[l1]) continue;
        if (D.mul_in[l1] % 16) return;
        const int n1 = 2 * l1 + 1;
        for (int p = D.pbeg[l1]; p < D.pend[l1]; ++p) {
            D.paths[p].b_off = words;
            words += tc_nkg(n1) * 64;
        }
        const int len = n1 * D.mul_in[l1];
        int stride = len;
        if (n1 == 1) { while (stride % 16 != 4) stride += 4; }
        else { while (stride % 32 != 8) stride += 4; }
        D.xs_off[l1] = xo;
        D.xs_stride[l1] = stride;
        xo += EC * stride;
    }
    D.nBF = words;
    D.xs_total = xo;
    if (conv_tc_smem_bytes(D, H) > 112 * 1024) return;
    struct Unit { int code, load; };
    std::vector<Unit> units;
    for (int l1 = 0; l1 <= D.lmax; ++l1) {
        if (!D.mul_in[l1] || D.pend[l1] <= D.pbeg[l1]) continue;
        const PathSets S = tc_path_sets(l1, D.lmax, D.kind);
        const int nkg = tc_nkg(2 * l1 + 1);
        for (int j = 0; j < S.n; ++j)
            for (int tile = 0; tile < D.mul_in[l1] / 16; ++tile)
                units.push_back({(l1 << 12) | (j << 8) | tile, (S.b[j + 1] - S.b[j]) * nkg + 2});
    }
    std::stable_sort(units.begin(), units.end(), [](const Unit& a, const Unit& b) { return a.load > b.load; });
    int load[CONV_WARPS] = {0}, cnt[CONV_WARPS] = {0};
    for (const Unit& u : units) {
        int best = -1;
        for (int w = 0; w < CONV_WARPS; ++w)
            if (cnt[w] < MAX_SLOTS_TC && (best < 0 || load[w] < load[best])) best = w;
        if (best < 0) return;
        D.slot_tc[best][cnt[best]++] = (int16_t)u.code;
        load[best] += u.load;
    }
    for (int w = 0; w < CONV_WARPS; ++w) D.n_slots_tc[w] = (int16_t)cnt[w];
    D.tc_ok = 1;
}

}  // namespace sn

using namespace sn;

// ---------------------------------------------------------------- workspace
namespace sn {

template <typename T>
static sevennet_status ws_alloc(Workspace* ws, T** p, int64_t count) {
    if (*p) {
        cudaFree(*p);
        ws->allocs.erase(std::remove(ws->allocs.begin(), ws->allocs.end(), (void*)*p), ws->allocs.end());
        *p = nullptr;
    }
    if (count <= 0) count = 1;
    void* q = nullptr;
    if (cudaMalloc(&q, (size_t)count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc of %lld bytes failed", (long long)(count * (int64_t)sizeof(T)));
        return SEVENNET_ENOMEM;
    }
    ws->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return SEVENNET_OK;
}

// Grows the workspace to the given sizes.  Nothing happens (and nothing waits)
// when the capacities suffice; a reallocation frees the old buffer first, and
// cudaFree waits for the work that may still use it.
sevennet_status ws_reserve(sevennet_model* M, Workspace* ws, int64_t n_atoms, int64_t n_edges,
                           int64_t n_bins, int64_t n_structs, cudaStream_t st) {
    (void)st;
    if (!ws->flags) {
        SN_TRY(ws_alloc(ws, &ws->flags, FLAG_WORDS));
        void* hp = nullptr;
        SN_CUDA(cudaMallocHost(&hp, FLAG_WORDS * sizeof(int)));
        ws->flags_host = static_cast<int*>(hp);
    }
    if (n_atoms > ws->cap_atoms) {
        const int64_t N = std::max<int64_t>(n_atoms, 16);
        const int T = M->T;
        SN_TRY(ws_alloc(ws, &ws->bin_of, N));
        SN_TRY(ws_alloc(ws, &ws->perm, N));
        SN_TRY(ws_alloc(ws, &ws->struct_of, N));
        SN_TRY(ws_alloc(ws, &ws->pos_s, N * 3));
        SN_TRY(ws_alloc(ws, &ws->frac_floor, N * 3));
        SN_TRY(ws_alloc(ws, &ws->q32, N));
        SN_TRY(ws_alloc(ws, &ws->species_s, N));
        SN_TRY(ws_alloc(ws, &ws->row_ptr, N + 1));
        SN_TRY(ws_alloc(ws, &ws->row_cnt, N + 1));
        SN_TRY(ws_alloc(ws, &ws->pair_ptr, N + 1));
        SN_TRY(ws_alloc(ws, &ws->h, N * M->h_max));
        SN_TRY(ws_alloc(ws, &ws->xs, (int64_t)T * N * M->x_max));
        SN_TRY(ws_alloc(ws, &ws->ys, (int64_t)T * N * M->y_max));
        SN_TRY(ws_alloc(ws, &ws->m, N * M->m_max));
        SN_TRY(ws_alloc(ws, &ws->gy, N * M->y_max));
        SN_TRY(ws_alloc(ws, &ws->gx, N * M->x_max));
        SN_TRY(ws_alloc(ws, &ws->gxq, N * M->x_max));
        SN_TRY(ws_alloc(ws, &ws->gh, N * M->h_max));
        SN_TRY(ws_alloc(ws, &ws->e_atom, N));
        SN_TRY(ws_alloc(ws, &ws->w_atom, N * 9));
        SN_TRY(ws_alloc(ws, &ws->f_s, N * 3));
        ws->cap_atoms = N;
    }
    if (n_edges > ws->cap_edges) {
        const int64_t E = std::max<int64_t>(n_edges, 1024);
        SN_CHECK(E < (1LL << 31) - 1, SEVENNET_EOVERFLOW, "edge count exceeds 2^31");
        SN_TRY(ws_alloc(ws, &ws->dst, E));
        SN_TRY(ws_alloc(ws, &ws->src, E));
        SN_TRY(ws_alloc(ws, &ws->shift, E * 3));
        SN_TRY(ws_alloc(ws, &ws->rev, E));
        SN_TRY(ws_alloc(ws, &ws->geom, E));
        SN_TRY(ws_alloc(ws, &ws->p_e, E));
        SN_TRY(ws_alloc(ws, &ws->p_dst, E));
        SN_TRY(ws_alloc(ws, &ws->p_src, E));
        SN_TRY(ws_alloc(ws, &ws->p_geom, E));
        SN_TRY(ws_alloc(ws, &ws->gd, E * 3));
        ws->cap_edges = E;
    }
    if (n_bins + 1 > ws->cap_bins) {
        const int64_t B = std::max<int64_t>(n_bins + 1, 64);
        SN_TRY(ws_alloc(ws, &ws->bin_count, B + 1));
        SN_TRY(ws_alloc(ws, &ws->bin_start, B + 1));
        SN_TRY(ws_alloc(ws, &ws->bin_fill, B + 1));
        ws->cap_bins = B;
    }
    if (n_structs > ws->cap_structs) {
        const int64_t S = std::max<int64_t>(n_structs, 4);
        SN_TRY(ws_alloc(ws, &ws->cells, S * 9));
        SN_TRY(ws_alloc(ws, &ws->inv_cells, S * 9));
        SN_TRY(ws_alloc(ws, &ws->sdesc, S * 16));
        SN_TRY(ws_alloc(ws, &ws->atom_off, S + 1));
        ws->cap_structs = S;
    }
    return SEVENNET_OK;
}

void ws_free(Workspace* ws) {
    if (!ws) return;
    for (void* p : ws->allocs) cudaFree(p);
    ws->allocs.clear();
    if (ws->flags_host) cudaFreeHost(ws->flags_host);
    delete ws;
}

// ---------------------------------------------------------------- evaluation
static void run_gemm(sevennet_model* M, const GemmBatch& g, sevennet_precision prec, cudaStream_t st) {
    if (!g.n) return;
    cudaEvent_t ev;
    prof_begin(&M->prof, PF_LINEAR, st, &ev);
    launch_gemm(g, prec, st);
    prof_end(&M->prof, PF_LINEAR, st, ev, 1);
    count_launches(1);
}

void model_embed(sevennet_model* M, Workspace* ws, int64_t N, cudaStream_t st) {
    cudaEvent_t ev;
    prof_begin(&M->prof, PF_OTHER, st, &ev);
    launch_embed(M->embed, ws->species_s, N, M->cfg.mul[0], M->cfg.n_species, ws->h, st);
    prof_end(&M->prof, PF_OTHER, st, ev, 1);
    count_launches(1);
}

// Block t forward on all N atoms: x = Lin1(h), y = LinSC(h); m = conv(x);
// y += Lin2(m); h = Gate(y).  x and y are kept for the adjoint.
void model_layer_forward(sevennet_model* M, Workspace* ws, int t, int64_t N, int64_t E,
                         sevennet_precision prec, cudaStream_t st) {
    const LayerDev& L = M->layers[t];
    Profiler* P = &M->prof;
    cudaEvent_t ev;
    float* x = ws->xs + (size_t)t * N * M->x_max;
    float* y = ws->ys + (size_t)t * N * M->y_max;
    GemmBatch g{};
    for (int l = 0; l < NL; ++l) {
        if (!L.in_mul[l]) continue;
        g.p[g.n++] = GemmProb{ws->h, L.lin1[l], L.lin1h[l], x, N, 2 * l + 1, L.in_mul[l], L.in_mul[l],
                              L.h_in_dim, L.in_off[l], L.x_dim, L.in_off[l], 0};
        if (L.y_mul[l])
            g.p[g.n++] = GemmProb{ws->h, L.sc[l], L.sch[l], y, N, 2 * l + 1, L.in_mul[l], L.y_mul[l],
                                  L.h_in_dim, L.in_off[l], L.y_dim, L.y_off[l], 0};
    }
    run_gemm(M, g, prec, st);
    prof_begin(P, PF_CONV_FWD, st, &ev);
    launch_conv_fwd(L, M->H, prec, N, E, ws->row_ptr, ws->dst, ws->src, ws->geom, x, ws->m, st, ws->flags);
    prof_end(P, PF_CONV_FWD, st, ev, 1);
    count_launches(1);
    GemmBatch g2{};
    for (int l = 0; l < NL; ++l) {
        if (!L.y_mul[l] || !L.msg_mul[l]) continue;
        g2.p[g2.n++] = GemmProb{ws->m, L.lin2[l], L.lin2h[l], y, N, 2 * l + 1, L.msg_mul[l], L.y_mul[l],
                                L.m_dim, L.msg_off[l], L.y_dim, L.y_off[l], L.in_mul[l] ? 1 : 0};
    }
    run_gemm(M, g2, prec, st);
    prof_begin(P, PF_GATE, st, &ev);
    launch_gate_fwd(L, M->cfg.mul[0], M->cfg.mul, M->lmax, N, y, ws->h, st);
    prof_end(P, PF_GATE, st, ev, 1);
    count_launches(1);
}

void model_readout(sevennet_model* M, Workspace* ws, int64_t N, cudaStream_t st) {
    cudaEvent_t ev;
    const int mul0 = M->cfg.mul[0];
    prof_begin(&M->prof, PF_OTHER, st, &ev);
    launch_readout(ws->h, M->layers[M->T - 1].h_out_dim, M->readout, M->shift_dev, ws->species_s, N, mul0,
                   M->cfg.n_species, ws->e_atom, st);
    prof_end(&M->prof, PF_OTHER, st, ev, 1);
    count_launches(1);
}

// Adjoint of the gate of block t: gy from gh (the last block takes the readout).
void model_layer_backward_gate(sevennet_model* M, Workspace* ws, int t, int64_t N, cudaStream_t st) {
    const LayerDev& L = M->layers[t];
    cudaEvent_t ev;
    float* y = ws->ys + (size_t)t * N * M->y_max;
    prof_begin(&M->prof, PF_GATE, st, &ev);
    launch_gate_bwd(L, M->cfg.mul[0], M->cfg.mul, M->lmax, N, y, ws->gh, M->readout, ws->gy, st);
    prof_end(&M->prof, PF_GATE, st, ev, 1);
    count_launches(1);
}

// The rest of the adjoint of block t: gm = Lin2^T(gy); conv adjoint (gx, and
// dE/dd accumulated into gd); for t > 0 gh = Lin1^T(gx) + LinSC^T(gy).
sevennet_status model_layer_backward_rest(sevennet_model* M, Workspace* ws, int t, int64_t N, int64_t E,
                                          sevennet_precision prec, cudaStream_t st, bool pairs) {
    const LayerDev& L = M->layers[t];
    cudaEvent_t ev;
    float* x = ws->xs + (size_t)t * N * M->x_max;
    GemmBatch g{};
    for (int l = 0; l < NL; ++l) {
        if (!L.y_mul[l] || !L.msg_mul[l]) continue;
        g.p[g.n++] = GemmProb{ws->gy, L.lin2T[l], L.lin2Th[l], ws->m, N, 2 * l + 1, L.y_mul[l], L.msg_mul[l],
                              L.y_dim, L.y_off[l], L.m_dim, L.msg_off[l], 0};
    }
    run_gemm(M, g, prec, st);
    prof_begin(&M->prof, PF_CONV_BWD, st, &ev);
    // the first block's dE/dx is not needed (its input is the species embedding)
    const int64_t bound = E < 0 ? ws->cap_edges : E;
    // a symmetric list has exactly E/2 pairs (a list that is not symmetric is an error the
    // reverse-edge build reports; the grid then covers the first of its pairs only)
    if (pairs)
        launch_conv_bwd_pair(L, M->H, prec, N, (bound + 1) / 2, ws->pair_ptr, ws->p_dst, ws->p_src, ws->p_geom,
                             ws->p_e, x, ws->m, t == 0 ? nullptr : ws->gx, ws->gxq, ws->flags, ws->gd, st);
    else
        launch_conv_bwd(L, M->H, prec, N, bound, ws->row_ptr, ws->dst, ws->src, ws->geom, x, ws->m,
                        t == 0 ? nullptr : ws->gx, ws->gxq, ws->flags, ws->gd, st);
    prof_end(&M->prof, PF_CONV_BWD, st, ev, t == 0 ? 1 : 2);
    count_launches(t == 0 ? 1 : 2);
    if (t == 0) return SEVENNET_OK;
    GemmBatch a{}, c{};
    for (int l = 0; l < NL; ++l) {
        if (!L.in_mul[l]) continue;
        a.p[a.n++] = GemmProb{ws->gx, L.lin1T[l], L.lin1Th[l], ws->gh, N, 2 * l + 1, L.in_mul[l], L.in_mul[l],
                              L.x_dim, L.in_off[l], L.h_in_dim, L.in_off[l], 0};
        if (L.y_mul[l])
            c.p[c.n++] = GemmProb{ws->gy, L.scT[l], L.scTh[l], ws->gh, N, 2 * l + 1, L.y_mul[l], L.in_mul[l],
                                  L.y_dim, L.y_off[l], L.h_in_dim, L.in_off[l], 1};
    }
    run_gemm(M, a, prec, st);
    run_gemm(M, c, prec, st);
    return SEVENNET_OK;
}

sevennet_status run_model(sevennet_model* M, Workspace* ws, const BatchHost& b, int64_t E,
                          sevennet_precision prec, double* energy_dev, double* forces_dev,
                          double* virial_dev, cudaStream_t st) {
    const int64_t N = b.atom_off[b.n_structs];
    const int T = M->T;
    cudaEvent_t ev;
    model_embed(M, ws, N, st);
    for (int t = 0; t < T; ++t) model_layer_forward(M, ws, t, N, E, prec, st);
    model_readout(M, ws, N, st);
    // reverse path (E < 0: the edge count is on the device; clear the capacity)
    const int64_t E_clear = E < 0 ? ws->cap_edges : E;
    if (E_clear > 0) SN_CUDA(cudaMemsetAsync(ws->gd, 0, (size_t)E_clear * 3 * sizeof(float), st));
    // the adjoint runs over unordered pairs of the (symmetric) neighbour list
    prof_begin(&M->prof, PF_NEIGHBORS, st, &ev);
    build_pairs(ws, N, st);
    prof_end(&M->prof, PF_NEIGHBORS, st, ev, 3);
    count_launches(3);
    for (int t = T - 1; t >= 0; --t) {
        model_layer_backward_gate(M, ws, t, N, st);
        SN_TRY(model_layer_backward_rest(M, ws, t, N, E, prec, st, true));
    }
    prof_begin(&M->prof, PF_OTHER, st, &ev);
    launch_forces(N, ws->row_ptr, ws->rev, ws->gd, ws->geom, ws->f_s, ws->w_atom, st);
    launch_reduce_structs(b.n_structs, ws->atom_off, ws->e_atom, ws->w_atom, energy_dev, virial_dev, st);
    launch_scatter_forces(N, ws->perm, ws->f_s, forces_dev, st);
    prof_end(&M->prof, PF_OTHER, st, ev, 3);
    count_launches(3);
    SN_CUDA(cudaGetLastError());
    return SEVENNET_OK;
}

}  // namespace sn

// ======================================================================= C ABI
extern "C" {

const char* sevennet_last_error(void) { return sn::g_last_error.c_str(); }

sevennet_status sevennet_padded_weights(const sevennet_model_config* cfg, const double* weights, size_t n_weights,
                                        int32_t* mul_out, double* out, size_t n_out) {
    std::string why;
    SN_CHECK(config_valid(cfg, &why), SEVENNET_EINVAL, "%s", why.c_str());
    const int64_t need = sevennet_n_params(cfg);
    SN_CHECK(weights && (int64_t)n_weights == need, SEVENNET_EINVAL,
             "weight vector has %zu entries, the model needs %lld", n_weights, (long long)need);
    sevennet_model_config pc;
    std::vector<double> wp;
    pad_model(cfg, &pc, weights, &wp);
    if (mul_out) for (int l = 0; l < 4; ++l) mul_out[l] = pc.mul[l];
    if (out) {
        SN_CHECK(n_out == wp.size(), SEVENNET_EINVAL, "output has %zu entries, the padded model has %zu", n_out,
                 wp.size());
        std::copy(wp.begin(), wp.end(), out);
    }
    return SEVENNET_OK;
}

int64_t sevennet_n_params(const sevennet_model_config* cfg) {
    std::string why;
    if (!config_valid(cfg, &why)) {
        set_error("%s", why.c_str());
        return -1;
    }
    auto e = weight_entries(cfg);
    return e.back().off + (int64_t)e.back().rows * e.back().cols;
}

sevennet_status sevennet_create_model(const sevennet_model_config* cfg, const double* weights,
                                      size_t n_weights, int device, sevennet_model** out) {
    SN_CHECK(out, SEVENNET_EINVAL, "out is NULL");
    *out = nullptr;
    std::string why;
    SN_CHECK(config_valid(cfg, &why), SEVENNET_EINVAL, "%s", why.c_str());
    const int64_t need = sevennet_n_params(cfg);
    SN_CHECK(weights && (int64_t)n_weights == need, SEVENNET_EINVAL,
             "weight vector has %zu entries, the model needs %lld", n_weights, (long long)need);
    for (size_t i = 0; i < n_weights; ++i)
        SN_CHECK(std::isfinite(weights[i]), SEVENNET_EINVAL, "weight %zu is not finite", i);
    // multiplicities that are not multiples of 32 run as the exact zero-padded model
    sevennet_model_config padded;
    std::vector<double> wpad;
    bool pad = false;
    for (int l = 0; l <= cfg->lmax; ++l) pad |= (cfg->mul[l] % 32) != 0;
    if (pad) {
        pad_model(cfg, &padded, weights, &wpad);
        cfg = &padded;
        weights = wpad.data();
    }
    int ndev = 0;
    SN_CUDA(cudaGetDeviceCount(&ndev));
    SN_CHECK(device >= 0 && device < ndev, SEVENNET_EINVAL, "device %d out of range (%d devices)", device, ndev);
    SN_ENTER(device);
    int major = 0, minor = 0;
    SN_CUDA(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device));
    SN_CUDA(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device));
    SN_CHECK(major == 10 && minor == 3, SEVENNET_EINVAL,
             "device %d is sm_%d%d; this library is built for sm_103a only", device, major, minor);

    auto* M = new sevennet_model();
    M->device = device;
    M->cfg = *cfg;
    M->shift.assign(cfg->n_species, 0.0);
    if (cfg->shift) for (int s = 0; s < cfg->n_species; ++s) M->shift[s] = cfg->shift[s];
    M->cfg.shift = nullptr;
    M->T = cfg->n_layers;
    M->lmax = cfg->lmax;
    M->H = cfg->mlp_hidden;
    M->NB = cfg->n_basis;
    auto fail = [&](sevennet_status s) { sevennet_destroy_model(M); return s; };

    auto entries = weight_entries(cfg);
    auto find = [&](const std::string& n) -> const WEntry* {
        for (auto& e : entries) if (e.name == n) return &e;
        return nullptr;
    };
    // embedding and readout
    {
        const WEntry* e = find("embed");
        std::vector<float> t((size_t)e->rows * e->cols);
        for (size_t i = 0; i < t.size(); ++i) t[i] = (float)weights[e->off + i];
        sevennet_status s = dev_upload(M, t, &M->embed);
        if (s) return fail(s);
        const WEntry* r0 = find("readout0");
        const WEntry* r1 = find("readout1");
        const int hid = cfg->readout_hidden;
        std::vector<float> c(cfg->mul[0]);
        for (int u = 0; u < cfg->mul[0]; ++u) {
            double acc = 0.0;
            for (int k = 0; k < hid; ++k) acc += weights[r0->off + (size_t)u * hid + k] * weights[r1->off + k];
            c[u] = (float)(cfg->scale * acc / std::sqrt((double)cfg->mul[0]) / std::sqrt((double)hid));
        }
        s = dev_upload(M, c, &M->readout);
        if (s) return fail(s);
        s = dev_upload(M, M->shift, &M->shift_dev);
        if (s) return fail(s);
    }
    const int H = cfg->mlp_hidden, NB = cfg->n_basis;
    M->layers.resize(M->T);
    for (int t = 0; t < M->T; ++t) {
        LayerDev& L = M->layers[t];
        std::vector<PathH> paths;
        block_irreps(cfg, t, L.in_mul, L.y_mul, L.out_mul, paths, L.msg_mul, &L.last);
        offsets(L.in_mul, L.in_off, &L.h_in_dim);
        offsets(L.y_mul, L.y_off, &L.y_dim);
        offsets(L.msg_mul, L.msg_off, &L.m_dim);
        offsets(L.out_mul, L.out_off, &L.h_out_dim);
        L.x_dim = L.h_in_dim;
        for (int l = 0; l < NL; ++l)
            if (L.y_mul[l] && !L.in_mul[l] && !L.msg_mul[l]) {
                set_error("block %d: gate input irrep %d has no producer", t);
                return fail(SEVENNET_EINVAL);
            }
        M->h_max = std::max({M->h_max, L.h_in_dim, L.h_out_dim});
        M->x_max = std::max(M->x_max, L.x_dim);
        M->y_max = std::max(M->y_max, L.y_dim);
        M->m_max = std::max(M->m_max, L.m_dim);
        // conv descriptor
        ConvDesc& D = L.conv;
        std::memset(&D, 0, sizeof(D));
        D.n_paths = (int)paths.size();
        if (D.n_paths > MAX_PATHS) { set_error("too many paths"); return fail(SEVENNET_EINVAL); }
        int col = 0, goff = 0;
        int ch[NL] = {};
        for (int l = 0; l < NL; ++l) { D.pbeg[l] = D.pend[l] = 0; }
        for (int p = 0; p < D.n_paths; ++p) {
            const PathH& q = paths[p];
            PathDesc& P = D.paths[p];
            P.l1 = q.l1; P.l2 = q.l2; P.l3 = q.l3;
            P.kind = coupling_kind(q.l1, q.l2, q.l3);
            P.mul = q.mul;
            P.col0 = col;
            P.x_off = L.in_off[q.l1];
            P.m_off = L.msg_off[q.l3];
            P.m_mul = L.msg_mul[q.l3];
            P.m_ch0 = ch[q.l3];
            P.g_off = goff;
            col += q.mul;
            ch[q.l3] += q.mul;
            goff += ((2 * q.l1 + 1) * (2 * q.l3 + 1) + 3) & ~3;   // 16-byte aligned G blocks
        }
        for (int l = 0; l < NL; ++l) {
            int b = -1, e = -1;
            for (int p = 0; p < D.n_paths; ++p)
                if (D.paths[p].l1 == l) { if (b < 0) b = p; e = p + 1; }
            D.pbeg[l] = b < 0 ? 0 : b;
            D.pend[l] = e < 0 ? 0 : e;
            D.mul_in[l] = L.in_mul[l];
            D.x_off[l] = L.in_off[l];
            if (L.in_mul[l]) D.l1max = l;
        }
        D.kind = (t == 0 ? 1 : 0) | (L.last ? 2 : 0);
        for (int l1 = 0; l1 <= MAX_LMAX; ++l1) {          // the kernels rely on this order
            const PathList pl = path_list(l1, cfg->lmax, D.kind);
            const int pb = path_begin(l1, cfg->lmax, D.kind);
            for (int i = 0; i < pl.n; ++i)
                if (pb + i >= D.n_paths || D.paths[pb + i].l1 != l1 || D.paths[pb + i].l2 != pl.l2[i] ||
                    D.paths[pb + i].l3 != pl.l3[i]) {
                    set_error("block %d: path table does not match the compile-time path list", t);
                    return fail(SEVENNET_EINVAL);
                }
        }
        D.W = col;
        D.Wpad = ((col + 3) & ~3) + 4;
        D.WpadB = ((col + 7) & ~7) + 8;
        D.H = H;
        D.n_basis = NB;
        D.lmax = cfg->lmax;
        D.ys = std::max(9, (cfg->lmax + 1) * (cfg->lmax + 1));
        D.x_dim = L.x_dim;
        D.m_dim = L.m_dim;
        D.nG = goff;
        D.r_cut = (float)cfg->r_cut;
        const double p = cfg->poly_p;
        D.env_a = (float)((p + 1.0) * (p + 2.0) / 2.0);
        D.env_b = (float)(p * (p + 2.0));
        D.env_c = (float)(p * (p + 1.0) / 2.0);
        D.poly_p = cfg->poly_p;
        if (!assign_slots(D, H)) { set_error("block %d: too many channel groups", t); return fail(SEVENNET_EINVAL); }
        assign_tc(D, H);
        // weights
        const std::string pre = "L" + std::to_string(t) + ".";
        sevennet_status s;
        for (int l = 0; l < NL; ++l) {
            if (L.in_mul[l]) {
                const WEntry* e = find(pre + "lin1." + std::to_string(l));
                s = upload_linear(M, weights + e->off, e->rows, e->cols, 1.0 / std::sqrt((double)e->rows),
                                  &L.lin1[l], &L.lin1T[l], &L.lin1h[l], &L.lin1Th[l]);
                if (s) return fail(s);
            }
            if (L.in_mul[l] && L.y_mul[l]) {
                const WEntry* e = find(pre + "sc." + std::to_string(l));
                s = upload_linear(M, weights + e->off, e->rows, e->cols, 1.0 / std::sqrt((double)e->rows),
                                  &L.sc[l], &L.scT[l], &L.sch[l], &L.scTh[l]);
                if (s) return fail(s);
            }
            if (L.msg_mul[l] && L.y_mul[l]) {
                const WEntry* e = find(pre + "lin2." + std::to_string(l));
                s = upload_linear(M, weights + e->off, e->rows, e->cols, 1.0 / std::sqrt((double)e->rows),
                                  &L.lin2[l], &L.lin2T[l], &L.lin2h[l], &L.lin2Th[l]);
                if (s) return fail(s);
            }
        }
        {
            const WEntry* e0 = find(pre + "mlp0");
            const WEntry* e1 = find(pre + "mlp1");
            const WEntry* e2 = find(pre + "mlp2");
            auto w0 = scaled(weights + e0->off, NB, H, 1.0 / std::sqrt((double)NB), false);
            auto w1 = scaled(weights + e1->off, H, H, 1.0 / std::sqrt((double)H), false);
            const double s2 = 1.0 / std::sqrt((double)H) / cfg->avg_num_neigh;
            auto w2 = scaled(weights + e2->off, H, D.W, s2, false);
            auto w2T = scaled(weights + e2->off, H, D.W, s2, true);
            if ((s = dev_upload(M, w0, &L.mlp0))) return fail(s);
            if ((s = dev_upload(M, w1, &L.mlp1))) return fail(s);
            auto w1T = scaled(weights + e1->off, H, H, 1.0 / std::sqrt((double)H), true);
            if ((s = dev_upload(M, w1T, &L.mlp1T))) return fail(s);
            if ((s = dev_upload(M, to_bf16_pair(w1), &L.mlp1h))) return fail(s);     // [k][j] hi, lo
            if ((s = dev_upload(M, to_bf16_pair(w1T), &L.mlp1Th))) return fail(s);   // [j][k] hi, lo
            if ((s = dev_upload(M, w2, &L.mlp2))) return fail(s);
            if ((s = dev_upload(M, w2T, &L.mlp2T))) return fail(s);
            if ((s = dev_upload(M, to_bf16(w2T), &L.mlp2h))) return fail(s);   // [W][H]
            if ((s = dev_upload(M, to_bf16(w2), &L.mlp2Th))) return fail(s);   // [H][W]
        }
    }
    sevennet_status s = conv_configure(H, M->layers);
    if (s) return fail(s);
    if (cudaStreamCreateWithFlags(&M->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaStreamCreate failed");
        return fail(SEVENNET_ECUDA);
    }
    M->ws = new Workspace();
    *out = M;
    return SEVENNET_OK;
}

void sevennet_destroy_model(sevennet_model* M) {
    if (!M) return;
    cudaSetDevice(M->device);
    if (M->stream) cudaStreamSynchronize(M->stream);
    ws_free(M->ws);
    for (void* p : M->allocations) cudaFree(p);
    if (M->stream) cudaStreamDestroy(M->stream);
    delete M;
}

}  // extern "C"

// ------------------------------------------------------------ neighbour lists
struct sevennet_nlist {
    int device;
    int64_t n_atoms, n_edges;
    int* dst = nullptr;    // input-order indices
    int* src = nullptr;
    int* shift = nullptr;
};

namespace sn {

sevennet_status check_batch(const BatchHost& b) {
    SN_CHECK(b.n_structs >= 1, SEVENNET_EINVAL, "n_structs must be >= 1");
    SN_CHECK(b.atom_off[0] == 0, SEVENNET_EINVAL, "atom_offsets[0] must be 0");
    for (int s = 0; s < b.n_structs; ++s)
        SN_CHECK(b.atom_off[s + 1] >= b.atom_off[s], SEVENNET_EINVAL, "atom_offsets must be non-decreasing");
    SN_CHECK(b.atom_off[b.n_structs] < (1LL << 30), SEVENNET_EINVAL, "too many atoms");
    for (double c : b.cells) SN_CHECK(std::isfinite(c), SEVENNET_EINVAL, "cell is not finite");
    return SEVENNET_OK;
}

__global__ void map_edges_kernel(int64_t E, const int* __restrict__ perm, const int* __restrict__ dst,
                                 const int* __restrict__ src, int* __restrict__ odst, int* __restrict__ osrc) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    odst[e] = perm[dst[e]];
    osrc[e] = perm[src[e]];
}

__global__ void check_species_kernel(int64_t n, const int32_t* __restrict__ sp, int ns, int* flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && (sp[i] < 0 || sp[i] >= ns)) atomicOr(flags + 3, 1);
}

// Enqueue the evaluation of a batch whose positions and species are on the
// device: neighbour build and model with the edge count kept on the device
// (no host synchronisation).  The edge capacity must have been reserved and the
// flags cleared; check_flags reads the outcome once the stream has reached it.
sevennet_status eval_enqueue(sevennet_model* M, Workspace* ws, const BatchHost& b,
                             const int32_t* species_dev, const double* pos_dev, sevennet_precision prec,
                             double* energy_dev, double* forces_dev, double* virial_dev, cudaStream_t st) {
    const int64_t N = b.atom_off[b.n_structs];
    int64_t E = -1;
    cudaEvent_t ev;
    prof_begin(&M->prof, PF_NEIGHBORS, st, &ev);
    SN_TRY(build_neighbors(M, ws, b, pos_dev, species_dev, st, &E, 0.0, nullptr, true));
    prof_end(&M->prof, PF_NEIGHBORS, st, ev, 10);
    count_launches(10);
    if (N > 0) {
        check_species_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, species_dev, M->cfg.n_species,
                                                                          ws->flags);
        count_launches(1);
    }
    return run_model(M, ws, b, E, prec, energy_dev, forces_dev, virial_dev, st);
}

sevennet_status check_flags(const int* f) {
    SN_CHECK(f[1] == 0, SEVENNET_EINVAL, "two atoms closer than 1e-8 A");
    SN_CHECK(f[3] == 0, SEVENNET_EINVAL, "species index out of range");
    SN_CHECK(f[FLAG_GX_OVERFLOW] == 0, SEVENNET_EOVERFLOW,
             "a feature gradient in the convolution adjoint reached 2^16 (outside the fixed-point range)");
    SN_CHECK(f[FLAG_EDGE_OVERFLOW] == 0, SEVENNET_EOVERFLOW, "neighbour list larger than its capacity");
    SN_CHECK(f[2] == 0, SEVENNET_ECUDA, "internal error: inconsistent neighbour list (a reverse edge not found, or a stored Verlet list entry out of range)");
    SN_CHECK(f[FLAG_COPY_TIMEOUT] == 0, SEVENNET_ETIMEDOUT, "a bulk copy did not complete within its bounded wait");
    return SEVENNET_OK;
}

// Edge capacity for a batch of N atoms: 64 neighbours per atom (the densest
// synthetic cells have about 50 within 5 A), grown to a larger count seen.
void reserve_edges(sevennet_model* M, Workspace* ws, int64_t N, int64_t need, sevennet_status* s) {
    const int64_t cap = std::max<int64_t>({ws->cap_edges, N * 64, need + need / 4 + 1024, 1024});
    *s = ws_reserve(M, ws, std::max<int64_t>(N, ws->cap_atoms), cap, ws->cap_bins - 1, ws->cap_structs,
                    nullptr);
}

// Evaluate a batch whose positions and species are already on the device: one
// host synchronisation, at the end; an overflow of the edge capacity is retried
// once with the count the device reported.
sevennet_status eval_batch(sevennet_model* M, Workspace* ws, const BatchHost& b,
                           const int32_t* species_dev, const double* pos_dev, sevennet_precision prec,
                           double* energy_dev, double* forces_dev, double* virial_dev, cudaStream_t st) {
    SN_TRY(check_batch(b));
    SN_CHECK(prec == SEVENNET_FP32 || prec == SEVENNET_BF16, SEVENNET_EINVAL, "unknown precision");
    const int64_t N = b.atom_off[b.n_structs];
    int64_t need = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        sevennet_status rs;
        reserve_edges(M, ws, N, need, &rs);
        SN_TRY(rs);
        SN_CUDA(cudaMemsetAsync(ws->flags, 0, FLAG_WORDS * sizeof(int), st));
        SN_TRY(eval_enqueue(M, ws, b, species_dev, pos_dev, prec, energy_dev, forces_dev, virial_dev, st));
        SN_CUDA(cudaMemcpyAsync(ws->flags_host, ws->flags, FLAG_WORDS * sizeof(int), cudaMemcpyDeviceToHost, st));
        SN_CUDA(cudaStreamSynchronize(st));
        if (ws->flags_host[FLAG_EDGE_OVERFLOW] && attempt == 0) {
            need = ws->flags_host[FLAG_EDGE_NEED];
            continue;
        }
        return check_flags(ws->flags_host);
    }
    return SEVENNET_OK;
}

}  // namespace sn

extern "C" {

sevennet_status sevennet_build_neighbors(sevennet_model* M, int64_t n_atoms, const double* pos,
                                         const double* cell, const int32_t pbc[3], sevennet_nlist** out,
                                         int64_t* n_edges) {
    SN_CHECK(M && out && n_edges && cell && (pos || n_atoms == 0), SEVENNET_EINVAL, "NULL argument");
    SN_CHECK(n_atoms >= 0, SEVENNET_EINVAL, "n_atoms < 0");
    *out = nullptr;
    SN_ENTER(M->device);
    BatchHost b;
    b.n_structs = 1;
    b.atom_off = {0, n_atoms};
    b.cells.assign(cell, cell + 9);
    b.pbc = {pbc ? pbc[0] : 1, pbc ? pbc[1] : 1, pbc ? pbc[2] : 1};
    SN_TRY(check_batch(b));
    for (int64_t i = 0; i < 3 * n_atoms; ++i) SN_CHECK(std::isfinite(pos[i]), SEVENNET_EINVAL, "position not finite");
    cudaStream_t st = M->stream;
    double* pos_dev = nullptr;
    int32_t* sp_dev = nullptr;
    SN_CUDA(cudaMallocAsync(&pos_dev, std::max<int64_t>(n_atoms, 1) * 3 * sizeof(double), st));
    SN_CUDA(cudaMallocAsync(&sp_dev, std::max<int64_t>(n_atoms, 1) * sizeof(int32_t), st));
    if (n_atoms) SN_CUDA(cudaMemcpyAsync(pos_dev, pos, n_atoms * 3 * sizeof(double), cudaMemcpyHostToDevice, st));
    SN_CUDA(cudaMemsetAsync(sp_dev, 0, std::max<int64_t>(n_atoms, 1) * sizeof(int32_t), st));
    int64_t E = 0;
    sevennet_status s = build_neighbors(M, M->ws, b, pos_dev, sp_dev, st, &E);
    if (s == SEVENNET_OK) {
        auto* nl = new sevennet_nlist();
        nl->device = M->device;
        nl->n_atoms = n_atoms;
        nl->n_edges = E;
        const size_t e1 = std::max<int64_t>(E, 1);
        if (cudaMalloc(&nl->dst, e1 * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&nl->src, e1 * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&nl->shift, e1 * 3 * sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            sevennet_nlist_destroy(nl);
            set_error("cudaMalloc failed for the neighbour list");
            s = SEVENNET_ENOMEM;
        } else {
            if (E > 0) {
                map_edges_kernel<<<(unsigned)((E + 255) / 256), 256, 0, st>>>(E, M->ws->perm, M->ws->dst,
                                                                              M->ws->src, nl->dst, nl->src);
                cudaMemcpyAsync(nl->shift, M->ws->shift, E * 3 * sizeof(int), cudaMemcpyDeviceToDevice, st);
            }
            if (cudaStreamSynchronize(st) != cudaSuccess) {
                set_error("neighbour list copy failed: %s", cudaGetErrorString(cudaGetLastError()));
                sevennet_nlist_destroy(nl);
                s = SEVENNET_ECUDA;
            } else {
                *out = nl;
                *n_edges = E;
            }
        }
    }
    cudaFreeAsync(pos_dev, st);
    cudaFreeAsync(sp_dev, st);
    return s;
}

sevennet_status sevennet_nlist_export(const sevennet_nlist* nl, int32_t* dst, int32_t* src, int32_t* shift) {
    SN_CHECK(nl, SEVENNET_EINVAL, "NULL list");
    SN_ENTER(nl->device);
    if (nl->n_edges == 0) return SEVENNET_OK;
    if (dst) SN_CUDA(cudaMemcpy(dst, nl->dst, nl->n_edges * sizeof(int), cudaMemcpyDeviceToHost));
    if (src) SN_CUDA(cudaMemcpy(src, nl->src, nl->n_edges * sizeof(int), cudaMemcpyDeviceToHost));
    if (shift) SN_CUDA(cudaMemcpy(shift, nl->shift, nl->n_edges * 3 * sizeof(int), cudaMemcpyDeviceToHost));
    return SEVENNET_OK;
}

void sevennet_nlist_destroy(sevennet_nlist* nl) {
    if (!nl) return;
    cudaSetDevice(nl->device);
    cudaFree(nl->dst);
    cudaFree(nl->src);
    cudaFree(nl->shift);
    delete nl;
}

sevennet_status sevennet_eval_energy_forces_virial(sevennet_model* M, int64_t n_atoms, const int32_t* species,
                                                   const double* pos, const double* cell, const int32_t pbc[3],
                                                   sevennet_precision prec, double* energy, double* forces,
                                                   double* virial) {
    SN_CHECK(M && cell && (n_atoms == 0 || (pos && species)), SEVENNET_EINVAL, "NULL argument");
    SN_CHECK(n_atoms >= 0, SEVENNET_EINVAL, "n_atoms < 0");
    SN_ENTER(M->device);
    for (int64_t i = 0; i < 3 * n_atoms; ++i) SN_CHECK(std::isfinite(pos[i]), SEVENNET_EINVAL, "position not finite");
    for (int64_t i = 0; i < n_atoms; ++i)
        SN_CHECK(species[i] >= 0 && species[i] < M->cfg.n_species, SEVENNET_EINVAL, "species index out of range");
    BatchHost b;
    b.n_structs = 1;
    b.atom_off = {0, n_atoms};
    b.cells.assign(cell, cell + 9);
    b.pbc = {pbc ? pbc[0] : 1, pbc ? pbc[1] : 1, pbc ? pbc[2] : 1};
    cudaStream_t st = M->stream;
    const size_t n1 = std::max<int64_t>(n_atoms, 1);
    double *pos_dev = nullptr, *f_dev = nullptr, *e_dev = nullptr, *w_dev = nullptr;
    int32_t* sp_dev = nullptr;
    SN_CUDA(cudaMallocAsync(&pos_dev, n1 * 3 * sizeof(double), st));
    SN_CUDA(cudaMallocAsync(&f_dev, n1 * 3 * sizeof(double), st));
    SN_CUDA(cudaMallocAsync(&sp_dev, n1 * sizeof(int32_t), st));
    SN_CUDA(cudaMallocAsync(&e_dev, 16 * sizeof(double), st));
    w_dev = e_dev + 4;
    if (n_atoms) {
        SN_CUDA(cudaMemcpyAsync(pos_dev, pos, n_atoms * 3 * sizeof(double), cudaMemcpyHostToDevice, st));
        SN_CUDA(cudaMemcpyAsync(sp_dev, species, n_atoms * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    }
    sevennet_status s = eval_batch(M, M->ws, b, sp_dev, pos_dev, prec, e_dev, f_dev, w_dev, st);
    if (s == SEVENNET_OK) {
        if (energy) cudaMemcpyAsync(energy, e_dev, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (virial) cudaMemcpyAsync(virial, w_dev, 9 * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (forces && n_atoms) cudaMemcpyAsync(forces, f_dev, n_atoms * 3 * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            set_error("result copy failed: %s", cudaGetErrorString(cudaGetLastError()));
            s = SEVENNET_ECUDA;
        }
    }
    cudaFreeAsync(pos_dev, st);
    cudaFreeAsync(f_dev, st);
    cudaFreeAsync(sp_dev, st);
    cudaFreeAsync(e_dev, st);
    cudaStreamSynchronize(st);
    return s;
}

sevennet_status sevennet_eval_batch_dev(sevennet_model* M, int32_t n_structs, const int64_t* atom_offsets,
                                        const double* cells, const int32_t* pbc, const int32_t* species_dev,
                                        const double* pos_dev, sevennet_precision prec, double* energy_dev,
                                        double* forces_dev, double* virial_dev, void* stream) {
    SN_CHECK(M && atom_offsets && cells && n_structs >= 1, SEVENNET_EINVAL, "bad argument");
    SN_ENTER(M->device);
    BatchHost b;
    b.n_structs = n_structs;
    b.atom_off.assign(atom_offsets, atom_offsets + n_structs + 1);
    b.cells.assign(cells, cells + (size_t)n_structs * 9);
    if (pbc) b.pbc.assign(pbc, pbc + (size_t)n_structs * 3);
    SN_CHECK(b.atom_off[n_structs] == 0 || (species_dev && pos_dev), SEVENNET_EINVAL, "NULL device array");
    cudaStream_t st = static_cast<cudaStream_t>(stream);   // NULL: the CUDA default stream
    return eval_batch(M, M->ws, b, species_dev, pos_dev, prec, energy_dev, forces_dev, virial_dev, st);
}

sevennet_status sevennet_conv_dims(const sevennet_model* M, int32_t layer, int32_t* x_dim, int32_t* m_dim) {
    SN_CHECK(M && layer >= 0 && layer < M->T, SEVENNET_EINVAL, "bad layer");
    if (x_dim) *x_dim = M->layers[layer].x_dim;
    if (m_dim) *m_dim = M->layers[layer].m_dim;
    return SEVENNET_OK;
}

sevennet_status sevennet_conv_forward_dev(sevennet_model* M, int32_t layer, int64_t n_atoms, int64_t n_edges,
                                          const int32_t* row_ptr, const int32_t* src, const float* d,
                                          const float* x, float* m_out, sevennet_precision prec, void* stream) {
    SN_CHECK(M && layer >= 0 && layer < M->T && n_atoms >= 0 && n_edges >= 0, SEVENNET_EINVAL, "bad argument");
    SN_CHECK(row_ptr && x && m_out && (n_edges == 0 || (src && d)), SEVENNET_EINVAL, "NULL argument");
    SN_ENTER(M->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);   // NULL: the CUDA default stream
    // build (dst, float4 geometry) from the caller's CSR + FP32 displacements
    int* dst = nullptr;
    float4* geom = nullptr;
    const size_t e1 = std::max<int64_t>(n_edges, 1);
    SN_CUDA(cudaMallocAsync(&dst, e1 * sizeof(int), st));
    SN_CUDA(cudaMallocAsync(&geom, e1 * sizeof(float4), st));
    conv_prepare_edges(n_atoms, n_edges, row_ptr, d, dst, geom, st);
    launch_conv_fwd(M->layers[layer], M->H, prec, n_atoms, n_edges, row_ptr, dst, src, geom, x, m_out, st);
    SN_CUDA(cudaGetLastError());
    cudaFreeAsync(dst, st);
    cudaFreeAsync(geom, st);
    return SEVENNET_OK;
}

sevennet_status sevennet_conv_backward_dev(sevennet_model* M, int32_t layer, int64_t n_atoms, int64_t n_edges,
                                           const int32_t* row_ptr, const int32_t* src, const float* d,
                                           const float* x, const float* g_m, float* g_x, float* g_d,
                                           sevennet_precision prec, void* stream) {
    SN_CHECK(M && layer >= 0 && layer < M->T && n_atoms >= 0 && n_edges >= 0, SEVENNET_EINVAL, "bad argument");
    SN_CHECK(row_ptr && x && g_m && g_x && (n_edges == 0 || (src && d && g_d)), SEVENNET_EINVAL, "NULL argument");
    SN_ENTER(M->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);   // NULL: the CUDA default stream
    int* dst = nullptr;
    float4* geom = nullptr;
    const size_t e1 = std::max<int64_t>(n_edges, 1);
    unsigned long long* gxq = nullptr;
    SN_CUDA(cudaMallocAsync(&dst, e1 * sizeof(int), st));
    SN_CUDA(cudaMallocAsync(&geom, e1 * sizeof(float4), st));
    SN_CUDA(cudaMallocAsync(&gxq, (size_t)std::max<int64_t>(n_atoms, 1) * M->layers[layer].x_dim *
                                      sizeof(unsigned long long), st));
    conv_prepare_edges(n_atoms, n_edges, row_ptr, d, dst, geom, st);
    launch_conv_bwd(M->layers[layer], M->H, prec, n_atoms, n_edges, row_ptr, dst, src, geom, x, g_m, g_x, gxq,
                    nullptr, g_d, st);
    SN_CUDA(cudaGetLastError());
    cudaFreeAsync(dst, st);
    cudaFreeAsync(geom, st);
    cudaFreeAsync(gxq, st);
    return SEVENNET_OK;
}

}  // extern "C"

extern "C" {

sevennet_status sevennet_profile(sevennet_model* M, int32_t enable) {
    SN_CHECK(M, SEVENNET_EINVAL, "NULL model");
    SN_ENTER(M->device);
    Profiler& p = M->prof;
    for (auto& r : p.pending) {
        cudaEventSynchronize(r.b);
        p.pool.push_back(r.a);
        p.pool.push_back(r.b);
    }
    p.pending.clear();
    for (int i = 0; i < PF_COUNT; ++i) { p.total_ms[i] = 0; p.launches[i] = 0; }
    p.on = enable != 0;
    return SEVENNET_OK;
}

sevennet_status sevennet_profile_read(sevennet_model* M, int32_t n_max, char* names, double* total_ms,
                                      int64_t* launches, int32_t* n_out) {
    SN_CHECK(M, SEVENNET_EINVAL, "NULL model");
    SN_ENTER(M->device);
    Profiler& p = M->prof;
    for (auto& r : p.pending) {
        SN_CUDA(cudaEventSynchronize(r.b));
        float ms = 0.f;
        SN_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
        p.total_ms[r.fam] += ms;
        p.pool.push_back(r.a);
        p.pool.push_back(r.b);
    }
    p.pending.clear();
    static const char* fam[PF_COUNT] = {"neighbors", "linear", "conv_fwd", "conv_bwd", "gate", "other"};
    const int n = std::min<int>(n_max, PF_COUNT);
    for (int i = 0; i < n; ++i) {
        if (names) { std::memset(names + 32 * i, 0, 32); std::strncpy(names + 32 * i, fam[i], 31); }
        if (total_ms) total_ms[i] = p.total_ms[i];
        if (launches) launches[i] = p.launches[i];
    }
    if (n_out) *n_out = n;
    return SEVENNET_OK;
}

int64_t sevennet_launch_count(void) { return g_launch_count.load(); }

}  // extern "C"
