// C ABI of the library: mesh, model and simulation handles, the window loop
// of Algorithm 1 on the host, and the device buffers it drives.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <limits>
#include <algorithm>
#include <map>
#include <tuple>
#include <memory>
#include <mutex>
#include <new>
#include <string>

#include "steps_internal.h"

using namespace steps;

namespace steps {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

}  // namespace steps

struct steps_mesh {
    HostMesh m;
};

struct steps_model {
    HostModel m;
};

namespace {

constexpr int kGraphWindows = 16;  // full windows per captured graph (even: buffer parity is restored)
constexpr int64_t kFlowTuneWindows = 72;  // windows the launch-form tuning takes (3 rounds of up to 3 groups)

__global__ void scatter_to_device_order(const int32_t *src, int64_t nt, int32_t S, const int32_t *inv_perm,
                                        int32_t *dst, size_t Tpad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    const int64_t d = inv_perm ? inv_perm[i] : i;
    for (int s = 0; s < S; ++s) dst[s * Tpad + d] = src[s * (size_t)nt + i];
}

__global__ void gather_to_original_order(const int32_t *src, int64_t nt, int32_t S, const int32_t *inv_perm,
                                         size_t Tpad, int32_t *dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    const int64_t d = inv_perm ? inv_perm[i] : i;
    for (int s = 0; s < S; ++s) dst[s * (size_t)nt + i] = src[s * Tpad + d];
}

__global__ void set_u64_kernel(uint64_t *p, uint64_t v) { *p = v; }

// *flag |= 1 if any of src[0..n) is negative (grid-stride; one atomic per warp at most)
__global__ void any_negative(const int32_t *src, int64_t n, uint32_t *flag) {
    bool neg = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        neg |= src[i] < 0;
    if (__any_sync(0xFFFFFFFFu, neg) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

// Launch-form choices of tuned simulations, shared by every simulation of
// the same compiled kernel, tet count and block size (clones of one
// prototype, the jobs of a stream): the first one's tuning run decides.
struct FlowChoice {
    int pick;
    float ms[3];
};
std::mutex g_flow_mu;
std::map<std::tuple<const void *, int64_t, int>, FlowChoice> g_flow_choice;

bool cuda_ok(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return true;
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return false;
}

}  // namespace

struct steps_sim {
    HostModel model;
    Tables tab;
    steps_options opt{};
    cudaStream_t stream = nullptr;
    int device = -1;                // the device current at creation (owns every buffer below)
    bool failed = false;            // a bounded device wait ran out: later runs are refused
    int64_t T = 0;
    int64_t Tpad = 0;
    int S = 0;
    uint64_t seed = 0;
    // device state
    int32_t *d_cnt[2] = {nullptr, nullptr};
    int cur = 0;
    int4 *d_nbr = nullptr;
    uint4 *d_thr = nullptr;
    float *d_inv_nav = nullptr;
    int32_t *d_orig = nullptr;      // device index -> original id (null without reordering)
    int32_t *d_inv_perm = nullptr;  // original id -> device index (null without reordering)
    uint32_t *d_rmask = nullptr;
    std::vector<uint32_t> h_rmask;  // device order
    uint32_t *d_err = nullptr;      // [2]: window error word, input check flag
    uint64_t *d_window_base = nullptr;
    int32_t *d_stage = nullptr;     // [S * nt] original-order staging
    int32_t *d_rec = nullptr;       // recording selection (species, then tets)
    size_t rec_bytes = 0;
    void *spec = nullptr;           // step kernel compiled for this model (cached process-wide), or null
    int32_t *d_trial = nullptr;     // [S][Tpad] trial counts for specialised kernels that keep them in global memory
    uint32_t *d_leave[2] = {nullptr, nullptr};  // EXP leave law: [S][Tpad] tables of the full and the last window
    std::string spec_why;           // why there is none
    // time
    double t_base = 0.0;
    int64_t k_grid = 0;
    uint64_t k_total = 0;
    uint64_t launches = 0;
    uint32_t scale_full[kMaxSpecies] = {};
    // graphs of kGraphWindows full windows, one per starting buffer
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    // flow launches (a run's full windows in one launch), per block size: [0]
    // the simulation's, [1] 512 (a tuning candidate when the block is smaller).
    // Each holds its step kernel, every tile's neighbour tiles (tiles of
    // `block` tets in device order, CSR), the tiles' finished-window words and
    // the item counter (d_flow[ntiles]).
    struct Flow {
        void *spec = nullptr;  // null with `generic`: the generic kernel's flow form (256-thread blocks)
        bool generic = false;
        int block = 0;
        bool tried = false;
        int32_t *d_tnb_off = nullptr;
        int32_t *d_tnb = nullptr;
        uint32_t *d_flow = nullptr;
        int64_t ntiles = 0;
        size_t bytes = 0;
    } flow[2];
    int flow_pick = -1;  // flow = 0 (tuned): -1 not yet timed, 0 window launches, 1 + k flow launches of flow[k]
    float flow_ms[3] = {0.f, 0.f, 0.f};  // tuning: ms per window of window launches, flow[0], flow[1]

    double time() const { return k_grid == 0 ? t_base : t_base + (double)k_grid * tab.tau; }

    ~steps_sim() {
        for (auto &g : graph)
            if (g) cudaGraphExecDestroy(g);
        cudaFree(d_cnt[0]);
        cudaFree(d_cnt[1]);
        cudaFree(d_nbr);
        cudaFree(d_thr);
        cudaFree(d_inv_nav);
        cudaFree(d_orig);
        cudaFree(d_inv_perm);
        cudaFree(d_rmask);
        cudaFree(d_err);
        cudaFree(d_window_base);
        cudaFree(d_stage);
        cudaFree(d_rec);
        cudaFree(d_trial);
        cudaFree(d_leave[0]);
        cudaFree(d_leave[1]);
        for (Flow &f : flow) {
            cudaFree(f.d_tnb_off);
            cudaFree(f.d_tnb);
            cudaFree(f.d_flow);
        }
    }

    // flow[k]'s kernel and tables (once): tile t lists itself and every tile
    // holding a face neighbour of one of its tets. flow[0] runs the
    // simulation's kernel (the generic one only at 256-thread blocks);
    // flow[1], 512-tet tiles of the specialised kernel, is compiled here. A
    // form without a kernel keeps no tables (d_flow null: no candidate).
    int ensure_flow(int k) {
        Flow &fl = flow[k];
        if (fl.d_flow || fl.tried) return STEPS_OK;
        fl.tried = true;
        const int64_t B = k == 0 ? opt.block : 512;
        void *sp = k == 0 ? spec : (spec ? spec_kernel(model, 512, nullptr) : nullptr);
        const bool generic = k == 0 && !spec;
        if (!sp && !(generic && B == 256)) return STEPS_OK;
        const int64_t nt = (T + B - 1) / B;
        std::vector<int32_t> off, nb, tmp;
        try {
            off.resize((size_t)nt + 1);
            for (int64_t t = 0; t < nt; ++t) {
                tmp.assign(1, (int32_t)t);
                for (int64_t d = t * B; d < std::min(T, (t + 1) * B); ++d)
                    for (int f = 0; f < 4; ++f) {
                        const int32_t j = tab.nbr_dev[(size_t)(4 * d + f)];
                        if (j >= 0 && j / B != t) tmp.push_back((int32_t)(j / B));
                    }
                std::sort(tmp.begin(), tmp.end());
                tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
                off[(size_t)t] = (int32_t)nb.size();
                nb.insert(nb.end(), tmp.begin(), tmp.end());
            }
            off[(size_t)nt] = (int32_t)nb.size();
        } catch (const std::bad_alloc &) {
            set_error("flow tables: out of host memory");
            return STEPS_ERR_OOM;
        }
        if (!cuda_ok(cudaMalloc((void **)&fl.d_tnb_off, off.size() * 4), "flow tables") ||
            !cuda_ok(cudaMalloc((void **)&fl.d_tnb, nb.size() * 4), "flow tables") ||
            !cuda_ok(cudaMalloc((void **)&fl.d_flow, ((size_t)nt + 1) * 4), "flow tables")) {
            cudaFree(fl.d_tnb_off);
            cudaFree(fl.d_tnb);
            cudaFree(fl.d_flow);
            fl.d_tnb_off = fl.d_tnb = nullptr;
            fl.d_flow = nullptr;
            return STEPS_ERR_OOM;
        }
        if (!cuda_ok(cudaMemcpy(fl.d_tnb_off, off.data(), off.size() * 4, cudaMemcpyHostToDevice), "flow tables") ||
            !cuda_ok(cudaMemcpy(fl.d_tnb, nb.data(), nb.size() * 4, cudaMemcpyHostToDevice), "flow tables") ||
            !cuda_ok(cudaMemset(fl.d_flow, 0, ((size_t)nt + 1) * 4), "flow tables"))
            return STEPS_ERR_CUDA;
        fl.spec = sp;
        fl.generic = generic;
        fl.block = (int)B;
        fl.ntiles = nt;
        fl.bytes = (off.size() + nb.size() + (size_t)nt + 1) * 4;
        return STEPS_OK;
    }

    // EXP leave law: the table of a window of length tau_k, into the full
    // window's buffer (tau_k == tau) or the last window's, in stream order
    // (the host copy is staged before the call returns)
    int upload_leave(double tau_k, cudaStream_t st) {
        if (!d_leave[0]) return STEPS_OK;
        std::vector<uint32_t> h;
        try {
            exp_leave_table(model, tab, tau_k, (size_t)Tpad, h);
        } catch (const std::bad_alloc &) {
            set_error("leave table: out of host memory");
            return STEPS_ERR_OOM;
        }
        uint32_t *dst = tau_k == tab.tau ? d_leave[0] : d_leave[1];
        return cuda_ok(cudaMemcpyAsync(dst, h.data(), h.size() * 4, cudaMemcpyHostToDevice, st), "leave table upload")
                   ? STEPS_OK
                   : STEPS_ERR_CUDA;
    }

    // the global trial buffer the model-specialised kernels of this model need (if any)
    int ensure_trial() {
        if (d_trial || !spec_global_trial(model)) return STEPS_OK;
        if (!cuda_ok(cudaMalloc((void **)&d_trial, (size_t)S * (size_t)Tpad * 4), "trial buffer"))
            return STEPS_ERR_OOM;
        drop_graphs();  // the captured launches hold the old arguments
        return STEPS_OK;
    }

    void drop_graphs() {
        for (auto &g : graph) {
            if (g) cudaGraphExecDestroy(g);
            g = nullptr;
        }
    }

    StepArgs args(int from, uint64_t window, const uint64_t *base, double tau_k, const uint32_t *scale) const {
        StepArgs a;
        std::memset(&a, 0, sizeof(a));
        a.cur = d_cnt[from];
        a.nxt = d_cnt[1 - from];
        a.nbr = d_nbr;
        a.thr = d_thr;
        a.inv_nav = d_inv_nav;
        a.orig = d_orig;
        a.rmask = d_rmask;
        a.err = d_err;
        a.T = (int32_t)T;
        a.Tpad = (int32_t)Tpad;
        a.key0 = (uint32_t)seed;
        a.key1 = (uint32_t)(seed >> 32);
        a.window = window;
        a.window_base = base;
        a.tau_k = tau_k;
        a.inv_tau_k = 1.0 / tau_k;
        a.tau_dn = (float)tau_k;
        if ((double)a.tau_dn > tau_k) a.tau_dn = std::nextafter(a.tau_dn, 0.0f);
        a.occ = opt.occupancy;
        a.prefetch = 1;  // the launch sets the distance: half a resident wave
        a.trial = d_trial;
        a.leave = d_leave[0] ? (tau_k == tab.tau ? d_leave[0] : d_leave[1]) : nullptr;
        std::memcpy(a.scale, scale, sizeof(a.scale));
        return a;
    }

    // one window on the model-specialised kernel if there is one, else the generic one
    int launch(const StepArgs &a, cudaStream_t st) const {
        return spec ? launch_spec(spec, model.dev, a, opt.block, st) : launch_step(model.dev, a, opt.block, st);
    }

    int window_launch(double tau_k) {  // one window of explicit length, plain launch
        uint32_t scale[kMaxSpecies] = {};
        for (int s = 0; s < S; ++s) scale[s] = species_scale(model, tab, s, tau_k);
        if (tau_k != tab.tau) {
            int rc = upload_leave(tau_k, stream);
            if (rc) return rc;
        }
        StepArgs a = args(cur, k_total, nullptr, tau_k, scale);
        int rc = launch(a, stream);
        if (rc) return rc;
        ++launches;
        cur = 1 - cur;
        ++k_total;
        return STEPS_OK;
    }

    int capture_graph(int from) {
        cudaStream_t cs = nullptr;
        if (!cuda_ok(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "cudaStreamCreate")) return STEPS_ERR_CUDA;
        int rc = STEPS_OK;
        cudaGraph_t g = nullptr;
        if (!cuda_ok(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture")) {
            cudaStreamDestroy(cs);
            return STEPS_ERR_CUDA;
        }
        int b = from;
        for (int q = 0; q < kGraphWindows && rc == STEPS_OK; ++q) {
            StepArgs a = args(b, (uint64_t)q, d_window_base, tab.tau, scale_full);
            rc = launch(a, cs);
            b = 1 - b;
        }
        if (rc == STEPS_OK) rc = launch_add_u64(d_window_base, kGraphWindows, cs);
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        if (rc == STEPS_OK && !cuda_ok(e, "cudaStreamEndCapture")) rc = STEPS_ERR_CUDA;
        if (rc == STEPS_OK && !cuda_ok(cudaGraphInstantiate(&graph[from], g, 0), "cudaGraphInstantiate"))
            rc = STEPS_ERR_CUDA;
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        return rc;
    }

    // a flow kernel exists for the simulation's block size
    bool flow_possible() const { return spec || opt.block == 256; }

    // n full windows: flow launches or window launches (all give the same bits)
    int full_windows(int64_t n) {
        if (opt.flow == 0 && flow_pick < 0 && flow_possible() && n >= kFlowTuneWindows) {
            int64_t used = 0;
            int rc = tune_flow(&used);
            if (rc) return rc;
            n -= used;
        }
        int k = -1;
        if (n >= 2 && flow_possible()) {
            if (opt.flow == 1) k = 0;
            else if (opt.flow == 0 && flow_pick >= 1) k = flow_pick - 1;
        }
        return k >= 0 ? flow_windows(n, k) : window_launches(n);
    }


    // The first run with enough full windows times the launch forms on
    // alternating groups of windows: window launches, flow launches at the
    // simulation's block size and, when that is below 512, flow launches of
    // 512-tet tiles. One warm round, so that one-time costs do not decide,
    // then two timed rounds, so that the state's slow drift cancels. The
    // fastest flow form is kept when it is more than 2 % faster than window
    // launches. The windows taken are ordinary windows of the run.
    int tune_flow(int64_t *used) {
        const auto key = std::make_tuple((const void *)spec, T, opt.block);
        {
            std::lock_guard<std::mutex> lock(g_flow_mu);
            auto it = g_flow_choice.find(key);
            if (it != g_flow_choice.end()) {
                flow_pick = it->second.pick;
                std::memcpy(flow_ms, it->second.ms, sizeof(flow_ms));
                return STEPS_OK;
            }
        }
        int rc = ensure_flow(0);
        if (!rc && opt.block < 512) rc = ensure_flow(1);
        if (rc) return rc;
        const int nc = flow[0].d_flow ? (flow[1].d_flow ? 3 : 2) : 1;
        if (nc == 1) {
            flow_pick = 0;
            return STEPS_OK;
        }
        cudaEvent_t e[4] = {};
        for (auto &ev : e)
            if (!cuda_ok(cudaEventCreate(&ev), "flow tuning event")) {
                for (auto &x : e)
                    if (x) cudaEventDestroy(x);
                return STEPS_ERR_CUDA;
            }
        float tot[3] = {0.f, 0.f, 0.f};
        const int64_t g = kFlowTuneWindows / (3 * nc);  // windows per group
        for (int round = 0; round < 3 && rc == STEPS_OK; ++round) {
            for (int c = 0; c < nc && rc == STEPS_OK; ++c) {
                if (!cuda_ok(cudaEventRecord(e[c], stream), "flow tuning")) rc = STEPS_ERR_CUDA;
                if (!rc) rc = c == 0 ? window_launches(g) : flow_windows(g, c - 1);
                *used += g;
            }
            if (!rc && !cuda_ok(cudaEventRecord(e[nc], stream), "flow tuning")) rc = STEPS_ERR_CUDA;
            if (!rc && !cuda_ok(cudaEventSynchronize(e[nc]), "flow tuning")) rc = STEPS_ERR_CUDA;
            for (int c = 0; c < nc && rc == STEPS_OK; ++c) {
                float ms = 0.f;
                if (!cuda_ok(cudaEventElapsedTime(&ms, e[c], e[c + 1]), "flow tuning")) rc = STEPS_ERR_CUDA;
                else if (round > 0) tot[c] += ms;
            }
        }
        for (auto &x : e) cudaEventDestroy(x);
        if (rc) return rc;
        int best = 1;
        for (int c = 2; c < nc; ++c)
            if (tot[c] < tot[best]) best = c;
        for (int c = 0; c < nc; ++c) flow_ms[c] = tot[c] / (2.f * (float)g);
        flow_pick = tot[best] < 0.98f * tot[0] ? best : 0;
        std::lock_guard<std::mutex> lock(g_flow_mu);
        FlowChoice ch;
        ch.pick = flow_pick;
        std::memcpy(ch.ms, flow_ms, sizeof(flow_ms));
        g_flow_choice[key] = ch;
        return STEPS_OK;
    }

    // n full windows, one launch each (graph replay of kGraphWindows at a time)
    int window_launches(int64_t n) {
        int64_t done = 0;
        if (opt.use_graph && n >= kGraphWindows) {
            if (!graph[cur]) {
                int rc = capture_graph(cur);
                if (rc) return rc;
            }
            set_u64_kernel<<<1, 1, 0, stream>>>(d_window_base, k_total);
            if (!cuda_ok(cudaGetLastError(), "set window base")) return STEPS_ERR_CUDA;
            ++launches;
            while (n - done >= kGraphWindows) {
                if (!cuda_ok(cudaGraphLaunch(graph[cur], stream), "cudaGraphLaunch")) return STEPS_ERR_CUDA;
                launches += kGraphWindows + 1;
                done += kGraphWindows;
                k_total += kGraphWindows;  // even: cur unchanged
            }
        }
        for (; done < n; ++done) {
            StepArgs a = args(cur, k_total, nullptr, tab.tau, scale_full);
            int rc = launch(a, stream);
            if (rc) return rc;
            ++launches;
            cur = 1 - cur;
            ++k_total;
        }
        return STEPS_OK;
    }

    // n full windows through launches of flow[k]'s kernel (one per 2^31 items)
    int flow_windows(int64_t n, int k) {
        int rc = ensure_flow(k);
        if (rc) return rc;
        const Flow &fl = flow[k];
        if (!fl.d_flow) return window_launches(n);
        const int64_t ntiles = fl.ntiles;
        uint32_t *const d_flow = fl.d_flow;
        const int64_t cap = std::max<int64_t>(1, (int64_t)0x7FFFFFFF / ntiles);
        for (int64_t done = 0; done < n;) {
            const int64_t nw = std::min(n - done, cap);
            if (!cuda_ok(cudaMemsetAsync(d_flow + ntiles, 0, 4, stream), "flow counter")) return STEPS_ERR_CUDA;
            StepArgs a = args(cur, k_total, nullptr, tab.tau, scale_full);
            FlowArgs f;
            f.tnb_off = fl.d_tnb_off;
            f.tnb = fl.d_tnb;
            f.tile_done = d_flow;
            f.fetch = d_flow + ntiles;
            f.nwin = (uint32_t)nw;
            f.ntiles = (uint32_t)ntiles;
            rc = fl.generic ? launch_flow(model.dev, a, f, fl.block, stream)
                            : launch_spec_flow(fl.spec, model.dev, a, f, fl.block, stream);
            if (rc) return rc;
            ++launches;
            done += nw;
            k_total += (uint64_t)nw;
            if (nw & 1) cur = 1 - cur;
        }
        return STEPS_OK;
    }
};

#define CHECK_NULL(p, name)                                    \
    do {                                                       \
        if (!(p)) {                                            \
            set_error(std::string(name) + ": NULL argument");  \
            return STEPS_ERR_ARG;                              \
        }                                                      \
    } while (0)

extern "C" {

const char *steps_last_error(void) { return g_last_error.c_str(); }

void steps_options_default(steps_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->occupancy = STEPS_OCC_MEAN;
    opt->reorder = STEPS_REORDER_MORTON;
    opt->block = 256;
    opt->use_graph = 1;
    opt->specialize = 0;
}

int steps_mesh_create(const double *verts_xyz, int64_t nv, const int32_t *tets, int64_t nt, steps_mesh **out) {
    CHECK_NULL(out, "steps_mesh_create");
    *out = nullptr;
    std::unique_ptr<steps_mesh> m(new (std::nothrow) steps_mesh);
    if (!m) {
        set_error("steps_mesh_create: out of host memory");
        return STEPS_ERR_OOM;
    }
    int rc;
    try {
        rc = build_mesh(verts_xyz, nv, tets, nt, m->m);
    } catch (const std::bad_alloc &) {
        set_error("steps_mesh_create: out of host memory");
        return STEPS_ERR_OOM;
    }
    if (rc) return rc;
    *out = m.release();
    return STEPS_OK;
}

void steps_mesh_destroy(steps_mesh *mesh) { delete mesh; }

int steps_mesh_num_tets(const steps_mesh *mesh, int64_t *nt) {
    CHECK_NULL(mesh, "steps_mesh_num_tets");
    CHECK_NULL(nt, "steps_mesh_num_tets");
    *nt = mesh->m.nt;
    return STEPS_OK;
}

int steps_model_create(int32_t n_species, const double *diff, int32_t n_reac, const int32_t *lhs,
                       const int32_t *rhs, const double *k, steps_model **out) {
    CHECK_NULL(out, "steps_model_create");
    *out = nullptr;
    std::unique_ptr<steps_model> m(new (std::nothrow) steps_model);
    if (!m) {
        set_error("steps_model_create: out of host memory");
        return STEPS_ERR_OOM;
    }
    int rc = build_model(n_species, diff, n_reac, lhs, rhs, k, m->m);
    if (rc) return rc;
    *out = m.release();
    return STEPS_OK;
}

void steps_model_destroy(steps_model *model) { delete model; }

int steps_sim_create(const steps_mesh *mesh, const steps_model *model, uint64_t seed, const steps_options *opt,
                     void *cuda_stream, steps_sim **out) {
    CHECK_NULL(out, "steps_sim_create");
    *out = nullptr;
    CHECK_NULL(mesh, "steps_sim_create");
    CHECK_NULL(model, "steps_sim_create");
    std::unique_ptr<steps_sim> s(new (std::nothrow) steps_sim);
    if (!s) {
        set_error("steps_sim_create: out of host memory");
        return STEPS_ERR_OOM;
    }
    if (opt) {
        s->opt = *opt;
        if (s->opt.block == 0) s->opt.block = 256;
        if (s->opt.block != 64 && s->opt.block != 128 && s->opt.block != 256 && s->opt.block != 512) {
            set_error("steps_sim_create: block must be 64, 128, 256 or 512");
            return STEPS_ERR_ARG;
        }
        if (s->opt.occupancy != STEPS_OCC_MEAN && s->opt.occupancy != STEPS_OCC_END) {
            set_error("steps_sim_create: bad occupancy mode");
            return STEPS_ERR_ARG;
        }
        if (s->opt.leave_law != STEPS_LEAVE_EULER && s->opt.leave_law != STEPS_LEAVE_EXP) {
            set_error("steps_sim_create: bad leave law");
            return STEPS_ERR_ARG;
        }
        if (s->opt.reorder != STEPS_REORDER_NONE && s->opt.reorder != STEPS_REORDER_MORTON &&
            s->opt.reorder != STEPS_REORDER_RCM) {
            set_error("steps_sim_create: bad reorder");
            return STEPS_ERR_ARG;
        }
        if (s->opt.flow < -1 || s->opt.flow > 1) {
            set_error("steps_sim_create: flow must be 0 (tuned), 1 (on) or -1 (off)");
            return STEPS_ERR_ARG;
        }
        if (s->opt.leave_law == STEPS_LEAVE_EXP) {
            if (s->opt.specialize < 0) {
                set_error("steps_sim_create: the EXP leave law runs on the model-specialised kernel only "
                          "(specialize must be 0 or 1)");
                return STEPS_ERR_ARG;
            }
            s->opt.specialize = 1;
        }
    } else {
        steps_options_default(&s->opt);
    }
    s->model = model->m;
    s->model.leave_exp = s->opt.leave_law == STEPS_LEAVE_EXP;
    s->stream = (cudaStream_t)cuda_stream;
    if (!cuda_ok(cudaGetDevice(&s->device), "steps_sim_create: cudaGetDevice")) return STEPS_ERR_CUDA;
    s->T = mesh->m.nt;
    s->Tpad = (s->T + 31) / 32 * 32;
    s->S = s->model.S;
    s->seed = seed;
    try {
        build_tables(mesh->m, s->model, s->opt.reorder, s->tab);
    } catch (const std::bad_alloc &) {
        set_error("steps_sim_create: out of host memory");
        return STEPS_ERR_OOM;
    }
    for (int sp = 0; sp < s->S; ++sp) s->scale_full[sp] = species_scale(s->model, s->tab, sp, s->tab.tau);

    const size_t T = (size_t)s->T, Tpad = (size_t)s->Tpad, S = (size_t)s->S;
    bool reordered = false;
    for (size_t d = 0; d < T && !reordered; ++d) reordered = s->tab.perm[d] != (int32_t)d;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    alloc((void **)&s->d_cnt[0], S * Tpad * 4);
    alloc((void **)&s->d_cnt[1], S * Tpad * 4);
    // per-tet tables are padded to Tpad entries (zeros) so that the step
    // kernel's bulk copies of a block's tile are whole multiples of 16 bytes
    alloc((void **)&s->d_nbr, Tpad * 16);
    alloc((void **)&s->d_thr, Tpad * 16);
    alloc((void **)&s->d_inv_nav, Tpad * 4);
    alloc((void **)&s->d_err, 8);
    alloc((void **)&s->d_window_base, 8);
    alloc((void **)&s->d_stage, S * T * 4);
    if (reordered) {
        alloc((void **)&s->d_orig, Tpad * 4);
        alloc((void **)&s->d_inv_perm, T * 4);
    }
    if (s->model.leave_exp) {
        alloc((void **)&s->d_leave[0], S * Tpad * 4);
        alloc((void **)&s->d_leave[1], S * Tpad * 4);
    }
    if (e != cudaSuccess) {
        set_error(std::string("steps_sim_create: device allocation failed: ") + cudaGetErrorString(e));
        cudaGetLastError();
        return STEPS_ERR_OOM;
    }
    bool ok = cuda_ok(cudaMemset(s->d_nbr, 0xFF, Tpad * 16), "memset") &&
              cuda_ok(cudaMemset(s->d_thr, 0, Tpad * 16), "memset") &&
              cuda_ok(cudaMemset(s->d_inv_nav, 0, Tpad * 4), "memset") &&
              cuda_ok(cudaMemcpy(s->d_nbr, s->tab.nbr_dev.data(), T * 16, cudaMemcpyHostToDevice), "upload nbr") &&
              cuda_ok(cudaMemcpy(s->d_thr, s->tab.thr_dev.data(), T * 16, cudaMemcpyHostToDevice), "upload thr") &&
              cuda_ok(cudaMemcpy(s->d_inv_nav, s->tab.inv_nav_dev.data(), T * 4, cudaMemcpyHostToDevice),
                      "upload inv_nav") &&
              cuda_ok(cudaMemset(s->d_cnt[0], 0, S * Tpad * 4), "memset") &&
              cuda_ok(cudaMemset(s->d_cnt[1], 0, S * Tpad * 4), "memset") &&
              cuda_ok(cudaMemset(s->d_err, 0, 8), "memset") && cuda_ok(cudaMemset(s->d_window_base, 0, 8), "memset");
    if (ok && reordered)
        ok = cuda_ok(cudaMemset(s->d_orig, 0, Tpad * 4), "memset") &&
             cuda_ok(cudaMemcpy(s->d_orig, s->tab.perm.data(), T * 4, cudaMemcpyHostToDevice), "upload perm") &&
             cuda_ok(cudaMemcpy(s->d_inv_perm, s->tab.inv_perm.data(), T * 4, cudaMemcpyHostToDevice),
                     "upload inv_perm");
    if (ok && s->model.leave_exp) {
        ok = s->upload_leave(s->tab.tau, s->stream) == STEPS_OK &&
             cuda_ok(cudaStreamSynchronize(s->stream), "leave table upload");
    }
    if (!ok) return STEPS_ERR_CUDA;
    // the model-specialised step kernel (compiled once per model and block size)
    constexpr int64_t kSpecializeMinTets = 65536;
    if (s->opt.specialize > 0 || (s->opt.specialize == 0 && s->T >= kSpecializeMinTets)) {
        s->spec = spec_kernel(s->model, s->opt.block, &s->spec_why);
        if (!s->spec && s->opt.specialize > 0) {
            set_error("steps_sim_create: the specialised step kernel could not be built: " + s->spec_why);
            return STEPS_ERR_CUDA;
        }
        if (s->spec) {
            int rc = s->ensure_trial();
            if (rc) return rc;
        }
    } else {
        s->spec_why = "not requested";
    }
    *out = s.release();
    return STEPS_OK;
}

int steps_sim_clone(const steps_sim *src, uint64_t seed, void *cuda_stream, steps_sim **out) {
    CHECK_NULL(out, "steps_sim_clone");
    *out = nullptr;
    CHECK_NULL(src, "steps_sim_clone");
    std::unique_ptr<steps_sim> s(new (std::nothrow) steps_sim);
    if (!s) {
        set_error("steps_sim_clone: out of host memory");
        return STEPS_ERR_OOM;
    }
    s->model = src->model;
    s->tab = src->tab;
    s->opt = src->opt;
    s->stream = (cudaStream_t)cuda_stream;
    s->device = src->device;
    s->T = src->T;
    s->Tpad = src->Tpad;
    s->S = src->S;
    s->seed = seed;
    s->h_rmask = src->h_rmask;
    s->spec = src->spec;
    s->spec_why = src->spec_why;
    std::memcpy(s->scale_full, src->scale_full, sizeof(s->scale_full));
    const size_t Tpad = (size_t)s->Tpad, S = (size_t)s->S, T = (size_t)s->T;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    alloc((void **)&s->d_cnt[0], S * Tpad * 4);
    alloc((void **)&s->d_cnt[1], S * Tpad * 4);
    alloc((void **)&s->d_nbr, Tpad * 16);
    alloc((void **)&s->d_thr, Tpad * 16);
    alloc((void **)&s->d_inv_nav, Tpad * 4);
    alloc((void **)&s->d_err, 8);
    alloc((void **)&s->d_window_base, 8);
    alloc((void **)&s->d_stage, S * T * 4);
    if (src->d_orig) {
        alloc((void **)&s->d_orig, Tpad * 4);
        alloc((void **)&s->d_inv_perm, T * 4);
    }
    if (src->d_rmask) alloc((void **)&s->d_rmask, Tpad * 4);
    if (src->d_trial) alloc((void **)&s->d_trial, S * Tpad * 4);
    if (src->d_leave[0]) {
        alloc((void **)&s->d_leave[0], S * Tpad * 4);
        alloc((void **)&s->d_leave[1], S * Tpad * 4);
    }
    if (e != cudaSuccess) {
        set_error(std::string("steps_sim_clone: device allocation failed: ") + cudaGetErrorString(e));
        cudaGetLastError();
        return STEPS_ERR_OOM;
    }
    cudaStream_t st = s->stream;
    bool ok = cuda_ok(cudaMemcpyAsync(s->d_nbr, src->d_nbr, Tpad * 16, cudaMemcpyDeviceToDevice, st), "clone") &&
              cuda_ok(cudaMemcpyAsync(s->d_thr, src->d_thr, Tpad * 16, cudaMemcpyDeviceToDevice, st), "clone") &&
              cuda_ok(cudaMemcpyAsync(s->d_inv_nav, src->d_inv_nav, Tpad * 4, cudaMemcpyDeviceToDevice, st), "clone") &&
              cuda_ok(cudaMemsetAsync(s->d_cnt[0], 0, S * Tpad * 4, st), "clone") &&
              cuda_ok(cudaMemsetAsync(s->d_cnt[1], 0, S * Tpad * 4, st), "clone") &&
              cuda_ok(cudaMemsetAsync(s->d_err, 0, 8, st), "clone") &&
              cuda_ok(cudaMemsetAsync(s->d_window_base, 0, 8, st), "clone");
    if (ok && src->d_orig)
        ok = cuda_ok(cudaMemcpyAsync(s->d_orig, src->d_orig, Tpad * 4, cudaMemcpyDeviceToDevice, st), "clone") &&
             cuda_ok(cudaMemcpyAsync(s->d_inv_perm, src->d_inv_perm, T * 4, cudaMemcpyDeviceToDevice, st), "clone");
    if (ok && src->d_rmask)
        ok = cuda_ok(cudaMemcpyAsync(s->d_rmask, src->d_rmask, Tpad * 4, cudaMemcpyDeviceToDevice, st), "clone");
    if (ok && src->d_leave[0])
        ok = cuda_ok(cudaMemcpyAsync(s->d_leave[0], src->d_leave[0], S * Tpad * 4, cudaMemcpyDeviceToDevice, st),
                     "clone");
    if (!ok || !cuda_ok(cudaStreamSynchronize(st), "steps_sim_clone")) return STEPS_ERR_CUDA;
    *out = s.release();
    return STEPS_OK;
}

int steps_sim_device_bytes(const steps_sim *sim, int64_t *bytes) {
    CHECK_NULL(sim, "steps_sim_device_bytes");
    CHECK_NULL(bytes, "steps_sim_device_bytes");
    const int64_t Tpad = sim->Tpad, S = sim->S, T = sim->T;
    *bytes = 2 * S * Tpad * 4 + Tpad * 16 * 2 + Tpad * 4 + 16 + S * T * 4 + (sim->d_orig ? Tpad * 4 + T * 4 : 0) +
             (sim->d_trial ? S * Tpad * 4 : 0) + (sim->d_leave[0] ? 2 * S * Tpad * 4 : 0) +
             (sim->d_rmask ? Tpad * 4 : 0) + (int64_t)(sim->flow[0].bytes + sim->flow[1].bytes);
    return STEPS_OK;
}

void steps_sim_destroy(steps_sim *sim) {
    if (!sim) return;
    if (sim->stream) cudaStreamSynchronize(sim->stream);
    else cudaDeviceSynchronize();
    delete sim;
}

static int put_counts(steps_sim *sim, int32_t s0, int32_t ns, const int32_t *counts) {
    const size_t T = (size_t)sim->T, Tpad = (size_t)sim->Tpad;
    if (!cuda_ok(cudaMemcpyAsync(sim->d_stage, counts, (size_t)ns * T * 4, cudaMemcpyHostToDevice, sim->stream),
                 "steps_set_counts: copy"))
        return STEPS_ERR_CUDA;
    // reject negative counts on the device, before anything of the state changes
    uint32_t neg = 0;
    const int64_t n = (int64_t)ns * (int64_t)T;
    if (!cuda_ok(cudaMemsetAsync(sim->d_err + 1, 0, 4, sim->stream), "steps_set_counts: check"))
        return STEPS_ERR_CUDA;
    any_negative<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, sim->stream>>>(sim->d_stage, n,
                                                                                               sim->d_err + 1);
    if (!cuda_ok(cudaGetLastError(), "steps_set_counts: check") ||
        !cuda_ok(cudaMemcpyAsync(&neg, sim->d_err + 1, 4, cudaMemcpyDeviceToHost, sim->stream), "steps_set_counts: check") ||
        !cuda_ok(cudaStreamSynchronize(sim->stream), "steps_set_counts: check"))
        return STEPS_ERR_CUDA;
    if (neg) {
        set_error("steps_set_counts: negative count");
        return STEPS_ERR_ARG;
    }
    scatter_to_device_order<<<(unsigned)((T + 255) / 256), 256, 0, sim->stream>>>(
        sim->d_stage, (int64_t)T, ns, sim->d_inv_perm, sim->d_cnt[sim->cur] + (size_t)s0 * Tpad, Tpad);
    if (!cuda_ok(cudaGetLastError(), "steps_set_counts: scatter")) return STEPS_ERR_CUDA;
    // the receiving buffer must start at zero (the step kernel writes only non-zero counts)
    if (!cuda_ok(cudaMemsetAsync(sim->d_cnt[1 - sim->cur] + (size_t)s0 * Tpad, 0, (size_t)ns * Tpad * 4,
                                 sim->stream),
                 "steps_set_counts: memset"))
        return STEPS_ERR_CUDA;
    if (!cuda_ok(cudaStreamSynchronize(sim->stream), "steps_set_counts")) return STEPS_ERR_CUDA;
    return STEPS_OK;
}


int steps_set_counts(steps_sim *sim, int32_t species, const int32_t *counts) {
    CHECK_NULL(sim, "steps_set_counts");
    CHECK_NULL(counts, "steps_set_counts");
    if (species < 0 || species >= sim->S) {
        set_error("steps_set_counts: species out of range");
        return STEPS_ERR_ARG;
    }
    return put_counts(sim, species, 1, counts);
}

int steps_set_counts_all(steps_sim *sim, const int32_t *counts) {
    CHECK_NULL(sim, "steps_set_counts_all");
    CHECK_NULL(counts, "steps_set_counts_all");
    return put_counts(sim, 0, sim->S, counts);
}

static int fetch_counts(const steps_sim *sim, int32_t s0, int32_t ns, int32_t *out) {
    const size_t T = (size_t)sim->T, Tpad = (size_t)sim->Tpad;
    gather_to_original_order<<<(unsigned)((T + 255) / 256), 256, 0, sim->stream>>>(
        sim->d_cnt[sim->cur] + (size_t)s0 * Tpad, (int64_t)T, ns, sim->d_inv_perm, Tpad, sim->d_stage);
    if (!cuda_ok(cudaGetLastError(), "steps_get_counts: gather")) return STEPS_ERR_CUDA;
    if (!cuda_ok(cudaMemcpyAsync(out, sim->d_stage, (size_t)ns * T * 4, cudaMemcpyDeviceToHost, sim->stream),
                 "steps_get_counts: copy"))
        return STEPS_ERR_CUDA;
    if (!cuda_ok(cudaStreamSynchronize(sim->stream), "steps_get_counts")) return STEPS_ERR_CUDA;
    return STEPS_OK;
}

int steps_get_counts(const steps_sim *sim, int32_t species, int32_t *out) {
    CHECK_NULL(sim, "steps_get_counts");
    CHECK_NULL(out, "steps_get_counts");
    if (species < 0 || species >= sim->S) {
        set_error("steps_get_counts: species out of range");
        return STEPS_ERR_ARG;
    }
    return fetch_counts(sim, species, 1, out);
}

int steps_get_counts_all(const steps_sim *sim, int32_t *out) {
    CHECK_NULL(sim, "steps_get_counts_all");
    CHECK_NULL(out, "steps_get_counts_all");
    return fetch_counts(sim, 0, sim->S, out);
}

int steps_set_reac_mask(steps_sim *sim, int32_t reac, const uint8_t *active) {
    CHECK_NULL(sim, "steps_set_reac_mask");
    if (reac < 0 || reac >= sim->model.R) {
        set_error("steps_set_reac_mask: reaction out of range");
        return STEPS_ERR_ARG;
    }
    const size_t T = (size_t)sim->T;
    if (sim->h_rmask.empty()) sim->h_rmask.assign(T, 0xFFFFFFFFu);
    const uint32_t bit = 1u << reac;
    for (size_t d = 0; d < T; ++d) {
        const bool on = !active || active[sim->tab.perm[d]] != 0;
        sim->h_rmask[d] = on ? (sim->h_rmask[d] | bit) : (sim->h_rmask[d] & ~bit);
    }
    if (!sim->d_rmask) {
        if (!cuda_ok(cudaMalloc((void **)&sim->d_rmask, (size_t)sim->Tpad * 4), "steps_set_reac_mask: alloc") ||
            !cuda_ok(cudaMemset(sim->d_rmask, 0, (size_t)sim->Tpad * 4), "steps_set_reac_mask: memset"))
            return STEPS_ERR_OOM;
        sim->drop_graphs();  // kernel arguments change
    }
    if (!cuda_ok(cudaStreamSynchronize(sim->stream), "steps_set_reac_mask") ||
        !cuda_ok(cudaMemcpy(sim->d_rmask, sim->h_rmask.data(), T * 4, cudaMemcpyHostToDevice),
                 "steps_set_reac_mask: copy"))
        return STEPS_ERR_CUDA;
    return STEPS_OK;
}

}  // extern "C"

namespace {

// A simulation whose bounded wait ran out stays closed: the block that gave up
// may have left a bulk copy in flight, so its results cannot be trusted.
int refuse_failed(const steps_sim *sim, const char *who) {
    if (!sim->failed) return STEPS_OK;
    set_error(std::string(who) + ": an earlier run of this simulation timed out on the device; "
                                 "destroy it and create a new one");
    return STEPS_ERR_STATE;
}

// Enqueues the windows of Algorithm 1 from the simulation's time to t_end
// (full windows of tau, then a shortened last window); no synchronisation.
int enqueue_run(steps_sim *sim, double t_end) {
    const double tau = sim->tab.tau;
    const bool finite = std::isfinite(tau);
    const double tol = finite ? 1e-9 * tau : 0.0;
    for (;;) {
        const double t = sim->time();
        if (!(t_end - t > tol)) break;
        if (finite && t + tau <= t_end + tol) {
            // the consecutive full windows the loop of Algorithm 1 takes from here
            int64_t n = 0;
            while (n < kWindowBatch) {
                const int64_t k = sim->k_grid + n;
                const double tt = k == 0 ? sim->t_base : sim->t_base + (double)k * tau;
                if (!(t_end - tt > tol) || !(tt + tau <= t_end + tol)) break;
                ++n;
            }
            int rc = sim->full_windows(n);
            if (rc) return rc;
            sim->k_grid += n;
        } else {
            int rc = sim->window_launch(t_end - t);  // shortened last window (Algorithm 1)
            if (rc) return rc;
            sim->t_base = t_end;
            sim->k_grid = 0;
            break;
        }
    }
    return STEPS_OK;
}

// Waits for the simulation's stream and turns the device error word into a
// return code (and clears it).
int finish_run(steps_sim *sim, const char *who) {
    uint32_t err = 0;
    if (!cuda_ok(cudaMemcpyAsync(&err, sim->d_err, 4, cudaMemcpyDeviceToHost, sim->stream), "error word") ||
        !cuda_ok(cudaStreamSynchronize(sim->stream), who))
        return STEPS_ERR_CUDA;
    if (err) {
        cudaMemsetAsync(sim->d_err, 0, 4, sim->stream);
        if (err & 4u) {
            sim->failed = true;
            set_error(std::string(who) + ": a bulk copy into shared memory did not complete within its wait limit; "
                                         "a copy may still be in flight, so this simulation is closed to further runs");
            return STEPS_ERR_TIMEOUT;
        }
        if (err & 8u) {
            sim->failed = true;
            set_error(std::string(who) + ": a tile of a flow launch waited beyond its limit for the tiles it depends "
                                         "on; the counts are not valid, so this simulation is closed to further runs");
            return STEPS_ERR_TIMEOUT;
        }
        set_error(std::string(who) + (err & 2u ? ": a tet fired more than 2^24 reactions in one window (rates too large)"
                                               : ": a negative count was seen on the device"));
        return STEPS_ERR_STATE;
    }
    return STEPS_OK;
}

// One recording: counts of the chosen species (rows of cur) at the chosen
// tets (device indices) into out[species][tet].
__global__ void gather_record(const int32_t *cur, size_t Tpad, const int32_t *species, int32_t ns,
                              const int32_t *tets, int32_t nr, int32_t *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)ns * nr) return;
    const int32_t q = (int32_t)(i / nr), j = (int32_t)(i % nr);
    out[i] = cur[(size_t)species[q] * Tpad + tets[j]];
}

}  // namespace

extern "C" {

int steps_run(steps_sim *sim, double t_end) {
    CHECK_NULL(sim, "steps_run");
    if (!std::isfinite(t_end)) {
        set_error("steps_run: t_end must be finite");
        return STEPS_ERR_ARG;
    }
    if (int rf = refuse_failed(sim, "steps_run")) return rf;
    int rc = enqueue_run(sim, t_end);
    return rc ? rc : finish_run(sim, "steps_run");
}

int steps_set_reac_rate(steps_sim *sim, int32_t reac, double k) {
    CHECK_NULL(sim, "steps_set_reac_rate");
    if (reac < 0 || reac >= sim->model.R) {
        set_error("steps_set_reac_rate: reaction out of range");
        return STEPS_ERR_ARG;
    }
    if (!(k >= 0.0) || !std::isfinite(k)) {
        set_error("steps_set_reac_rate: rate constant must be finite and >= 0");
        return STEPS_ERR_ARG;
    }
    sim->model.k[(size_t)reac] = k;
    sim->model.dev.reac[reac].k = (float)k;
    sim->drop_graphs();  // the captured launches hold the old model
    return STEPS_OK;
}

int steps_run_record(steps_sim *sim, double t_end, double dt_rec, int32_t n_species, const int32_t *species,
                     int32_t n_tets, const int32_t *tets, int32_t *d_out, int64_t max_records, int64_t *n_records) {
    CHECK_NULL(sim, "steps_run_record");
    CHECK_NULL(species, "steps_run_record");
    CHECK_NULL(tets, "steps_run_record");
    CHECK_NULL(d_out, "steps_run_record");
    if (n_records) *n_records = 0;
    if (!std::isfinite(t_end) || !(dt_rec > 0.0) || !std::isfinite(dt_rec)) {
        set_error("steps_run_record: t_end must be finite and dt_rec finite and > 0");
        return STEPS_ERR_ARG;
    }
    if (int rf = refuse_failed(sim, "steps_run_record")) return rf;
    if (n_species < 1 || n_species > sim->S || n_tets < 1 || max_records < 0) {
        set_error("steps_run_record: bad species or tet count");
        return STEPS_ERR_ARG;
    }
    for (int32_t q = 0; q < n_species; ++q)
        if (species[q] < 0 || species[q] >= sim->S) {
            set_error("steps_run_record: species out of range");
            return STEPS_ERR_ARG;
        }
    std::vector<int32_t> dev_tets((size_t)n_tets);
    for (int32_t j = 0; j < n_tets; ++j) {
        if (tets[j] < 0 || tets[j] >= sim->T) {
            set_error("steps_run_record: tet out of range");
            return STEPS_ERR_ARG;
        }
        dev_tets[(size_t)j] = sim->tab.inv_perm.empty() ? tets[j] : sim->tab.inv_perm[(size_t)tets[j]];
    }
    // recording times t0 + k dt_rec, k = 1, 2, ... up to t_end (recomputed, not accumulated)
    const double t0 = sim->time();
    const double tol = 1e-12 * std::max(std::fabs(t_end), dt_rec);
    int64_t nrec = 0;
    while (t0 + (double)(nrec + 1) * dt_rec <= t_end + tol) ++nrec;
    if (nrec > max_records) {
        set_error("steps_run_record: " + std::to_string(nrec) + " recordings do not fit max_records = " +
                  std::to_string(max_records));
        return STEPS_ERR_ARG;
    }
    // the selection, uploaded once
    const size_t need = ((size_t)n_species + (size_t)n_tets) * 4;
    if (sim->rec_bytes < need) {
        cudaFree(sim->d_rec);
        sim->d_rec = nullptr;
        sim->rec_bytes = 0;
        if (!cuda_ok(cudaMalloc((void **)&sim->d_rec, need), "steps_run_record: alloc")) return STEPS_ERR_OOM;
        sim->rec_bytes = need;
    }
    int32_t *d_species = sim->d_rec, *d_tets = sim->d_rec + n_species;
    if (!cuda_ok(cudaMemcpyAsync(d_species, species, (size_t)n_species * 4, cudaMemcpyHostToDevice, sim->stream),
                 "steps_run_record: upload") ||
        !cuda_ok(cudaMemcpyAsync(d_tets, dev_tets.data(), (size_t)n_tets * 4, cudaMemcpyHostToDevice, sim->stream),
                 "steps_run_record: upload"))
        return STEPS_ERR_CUDA;
    const int64_t per = (int64_t)n_species * n_tets;
    const unsigned grid = (unsigned)((per + 255) / 256);
    for (int64_t k = 1; k <= nrec; ++k) {
        int rc = enqueue_run(sim, t0 + (double)k * dt_rec);
        if (rc) return rc;
        gather_record<<<grid, 256, 0, sim->stream>>>(sim->d_cnt[sim->cur], (size_t)sim->Tpad, d_species, n_species,
                                                     d_tets, n_tets, d_out + (k - 1) * per);
        if (!cuda_ok(cudaGetLastError(), "steps_run_record: gather")) return STEPS_ERR_CUDA;
        ++sim->launches;
    }
    int rc = enqueue_run(sim, t_end);
    if (!rc) rc = finish_run(sim, "steps_run_record");
    // the host copy of dev_tets must outlive the async upload: finish_run synchronised
    if (n_records) *n_records = rc ? 0 : nrec;
    return rc;
}

int steps_sim_flow(const steps_sim *sim, int32_t *flow_block, float *tune_ms) {
    CHECK_NULL(sim, "steps_sim_flow");
    CHECK_NULL(flow_block, "steps_sim_flow");
    int k = -1;
    if (sim->flow_possible()) {
        if (sim->opt.flow == 1) k = 0;
        else if (sim->opt.flow == 0 && sim->flow_pick >= 1) k = sim->flow_pick - 1;
    }
    *flow_block = k < 0 ? 0 : k == 0 ? sim->opt.block : 512;
    if (tune_ms)
        for (int c = 0; c < 3; ++c) tune_ms[c] = sim->flow_ms[c];
    return STEPS_OK;
}

int steps_sim_specialized(const steps_sim *sim, int32_t *specialized) {
    CHECK_NULL(sim, "steps_sim_specialized");
    CHECK_NULL(specialized, "steps_sim_specialized");
    *specialized = sim->spec ? 1 : 0;
    return STEPS_OK;
}

int steps_get_time(const steps_sim *sim, double *t) {
    CHECK_NULL(sim, "steps_get_time");
    CHECK_NULL(t, "steps_get_time");
    *t = sim->time();
    return STEPS_OK;
}

int steps_get_tau(const steps_sim *sim, double *tau) {
    CHECK_NULL(sim, "steps_get_tau");
    CHECK_NULL(tau, "steps_get_tau");
    *tau = sim->tab.tau;
    return STEPS_OK;
}

int steps_sim_shape(const steps_sim *sim, int64_t *nt, int32_t *n_species) {
    CHECK_NULL(sim, "steps_sim_shape");
    if (nt) *nt = sim->T;
    if (n_species) *n_species = sim->S;
    return STEPS_OK;
}

int steps_get_windows(const steps_sim *sim, uint64_t *windows, uint64_t *launches) {
    CHECK_NULL(sim, "steps_get_windows");
    if (windows) *windows = sim->k_total;
    if (launches) *launches = sim->launches;
    return STEPS_OK;
}

int steps_debug_philox(uint64_t seed, const uint32_t *ctr, int64_t n, uint32_t *out) {
    CHECK_NULL(ctr, "steps_debug_philox");
    CHECK_NULL(out, "steps_debug_philox");
    if (n < 0) return STEPS_ERR_ARG;
    if (n == 0) return STEPS_OK;
    uint32_t *dc = nullptr, *dout = nullptr;
    int rc = STEPS_OK;
    if (!cuda_ok(cudaMalloc((void **)&dc, (size_t)n * 16), "alloc") ||
        !cuda_ok(cudaMalloc((void **)&dout, (size_t)n * 16), "alloc"))
        rc = STEPS_ERR_OOM;
    if (!rc && !cuda_ok(cudaMemcpy(dc, ctr, (size_t)n * 16, cudaMemcpyHostToDevice), "copy")) rc = STEPS_ERR_CUDA;
    if (!rc) rc = launch_philox_test(seed, dc, n, dout, nullptr);
    if (!rc && !cuda_ok(cudaMemcpy(out, dout, (size_t)n * 16, cudaMemcpyDeviceToHost), "copy")) rc = STEPS_ERR_CUDA;
    cudaFree(dc);
    cudaFree(dout);
    return rc;
}

int steps_debug_host_tables(const steps_mesh *mesh, const steps_model *model, int32_t reorder, double *tau,
                            uint32_t *thr, int32_t *perm) {
    CHECK_NULL(mesh, "steps_debug_host_tables");
    CHECK_NULL(model, "steps_debug_host_tables");
    CHECK_NULL(tau, "steps_debug_host_tables");
    CHECK_NULL(thr, "steps_debug_host_tables");
    if (reorder != STEPS_REORDER_NONE && reorder != STEPS_REORDER_MORTON && reorder != STEPS_REORDER_RCM) {
        set_error("steps_debug_host_tables: bad reorder");
        return STEPS_ERR_ARG;
    }
    Tables t;
    try {
        build_tables(mesh->m, model->m, reorder, t);
    } catch (const std::bad_alloc &) {
        set_error("steps_debug_host_tables: out of host memory");
        return STEPS_ERR_OOM;
    }
    *tau = t.tau;
    const size_t nt = t.perm.size();
    for (size_t d = 0; d < nt; ++d)
        for (int f = 0; f < 4; ++f) thr[(size_t)t.perm[d] * 4 + f] = t.thr_dev[d * 4 + f];
    if (perm) std::memcpy(perm, t.perm.data(), nt * sizeof(int32_t));
    return STEPS_OK;
}

int steps_debug_wait(int32_t deliver, int64_t limit_cycles) {
    if (limit_cycles < 1 || limit_cycles > (int64_t)1 << 31) {
        set_error("steps_debug_wait: limit_cycles must be in [1, 2^31]");
        return STEPS_ERR_ARG;
    }
    void *src = nullptr;
    uint32_t *status = nullptr;
    int rc = STEPS_OK;
    if (!cuda_ok(cudaMalloc(&src, 16), "steps_debug_wait: alloc") ||
        !cuda_ok(cudaMalloc((void **)&status, 4), "steps_debug_wait: alloc"))
        rc = STEPS_ERR_OOM;
    uint32_t st = 0;
    if (!rc && (!cuda_ok(cudaMemset(src, 0, 16), "steps_debug_wait") ||
                !cuda_ok(cudaMemset(status, 0xFF, 4), "steps_debug_wait")))
        rc = STEPS_ERR_CUDA;
    if (!rc) rc = launch_wait_test(src, deliver != 0, (long long)limit_cycles, status, nullptr);
    if (!rc && !cuda_ok(cudaMemcpy(&st, status, 4, cudaMemcpyDeviceToHost), "steps_debug_wait")) rc = STEPS_ERR_CUDA;
    cudaFree(src);
    cudaFree(status);
    if (rc) return rc;
    if (st == 4u) {
        set_error("steps_debug_wait: the bulk-copy wait did not complete within its limit");
        return STEPS_ERR_TIMEOUT;
    }
    if (st != 0u) {
        set_error("steps_debug_wait: unexpected status");
        return STEPS_ERR_STATE;
    }
    return STEPS_OK;
}

int steps_debug_flow_wait(int32_t deliver, int64_t limit_cycles) {
    if (limit_cycles < 1 || limit_cycles > (int64_t)1 << 31) {
        set_error("steps_debug_flow_wait: limit_cycles must be in [1, 2^31]");
        return STEPS_ERR_ARG;
    }
    // tile 0 lists 40 neighbour tiles (two rounds of the warp); all of them
    // have finished window 4 (word 5) when delivered, else the last has not
    constexpr int n = 40;
    int32_t h_off[2] = {0, n}, h_nb[n];
    uint32_t h_done[n];
    for (int j = 0; j < n; ++j) {
        h_nb[j] = j;
        h_done[j] = 5u + (uint32_t)(j % 3);
    }
    if (!deliver) h_done[n - 1] = 4u;
    int32_t *d_off = nullptr, *d_nb = nullptr;
    uint32_t *d_done = nullptr, *status = nullptr;
    int rc = STEPS_OK;
    if (!cuda_ok(cudaMalloc((void **)&d_off, sizeof(h_off)), "steps_debug_flow_wait: alloc") ||
        !cuda_ok(cudaMalloc((void **)&d_nb, sizeof(h_nb)), "steps_debug_flow_wait: alloc") ||
        !cuda_ok(cudaMalloc((void **)&d_done, sizeof(h_done)), "steps_debug_flow_wait: alloc") ||
        !cuda_ok(cudaMalloc((void **)&status, 4), "steps_debug_flow_wait: alloc"))
        rc = STEPS_ERR_OOM;
    uint32_t st = 0;
    if (!rc && (!cuda_ok(cudaMemcpy(d_off, h_off, sizeof(h_off), cudaMemcpyHostToDevice), "steps_debug_flow_wait") ||
                !cuda_ok(cudaMemcpy(d_nb, h_nb, sizeof(h_nb), cudaMemcpyHostToDevice), "steps_debug_flow_wait") ||
                !cuda_ok(cudaMemcpy(d_done, h_done, sizeof(h_done), cudaMemcpyHostToDevice), "steps_debug_flow_wait") ||
                !cuda_ok(cudaMemset(status, 0xFF, 4), "steps_debug_flow_wait")))
        rc = STEPS_ERR_CUDA;
    if (!rc) rc = launch_flow_wait_test(d_off, d_nb, d_done, (long long)limit_cycles, status);
    if (!rc && !cuda_ok(cudaMemcpy(&st, status, 4, cudaMemcpyDeviceToHost), "steps_debug_flow_wait"))
        rc = STEPS_ERR_CUDA;
    cudaFree(d_off);
    cudaFree(d_nb);
    cudaFree(d_done);
    cudaFree(status);
    if (rc) return rc;
    if (st == 8u) {
        set_error("steps_debug_flow_wait: the dependency wait did not complete within its limit");
        return STEPS_ERR_TIMEOUT;
    }
    if (st != 0u) {
        set_error("steps_debug_flow_wait: unexpected status");
        return STEPS_ERR_STATE;
    }
    return STEPS_OK;
}

int steps_debug_logf(const float *x, int64_t n, float *out) {
    CHECK_NULL(x, "steps_debug_logf");
    CHECK_NULL(out, "steps_debug_logf");
    if (n < 0) return STEPS_ERR_ARG;
    if (n == 0) return STEPS_OK;
    float *dx = nullptr, *dout = nullptr;
    int rc = STEPS_OK;
    if (!cuda_ok(cudaMalloc((void **)&dx, (size_t)n * 4), "alloc") ||
        !cuda_ok(cudaMalloc((void **)&dout, (size_t)n * 4), "alloc"))
        rc = STEPS_ERR_OOM;
    if (!rc && !cuda_ok(cudaMemcpy(dx, x, (size_t)n * 4, cudaMemcpyHostToDevice), "copy")) rc = STEPS_ERR_CUDA;
    if (!rc) rc = launch_logf_test(dx, n, dout, nullptr);
    if (!rc && !cuda_ok(cudaMemcpy(out, dout, (size_t)n * 4, cudaMemcpyDeviceToHost), "copy")) rc = STEPS_ERR_CUDA;
    cudaFree(dx);
    cudaFree(dout);
    return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched form: one launch per window over many simulations.
// ---------------------------------------------------------------------------
struct steps_batch {
    std::vector<steps_sim *> members;
    cudaStream_t stream = nullptr;
    int block = 256;
    bool autotune = false;
    bool use_graph = true;
    int max_S = 1, max_R = 0;
    bool any_order0 = false;
    RepEntry *h_reps = nullptr;  // pinned host mirror (full windows)
    RepEntry *h_last = nullptr;  // pinned host table of the shortened last windows: a second buffer, so
                                 // that filling it cannot change h_reps while its upload is still queued
    RepEntry *d_reps = nullptr;
    uint32_t *d_err = nullptr;
    uint32_t *h_err = nullptr;   // pinned copy of the error word, read after the stream completes
    struct Work {
        BlockWork *d = nullptr;
        int64_t n = 0;
        cudaGraphExec_t graph = nullptr;
    };
    Work work[4];  // block sizes 64, 128, 256, 512
    uint64_t launches = 0;
    bool use_spec = false;      // run the model-specialised batched kernel
    bool spec_forced = false;
    void *spec[4] = {};         // per block size, compiled on first use (before any capture)
    std::string spec_why;
    std::vector<float> tune_ms;  // autotune timings per candidate block (ms per window)
    bool flow = false;           // full windows of member groups as flow launches (specialised kernel)
    // flow launches, per block size: the neighbour tiles of every work entry
    // (CSR over work indices), the entries' finished-window words followed by
    // the item counter, and the groups: consecutive members whose tables fit
    // in about half of L2 (at least one member each), so that a group's
    // windows run from L2
    struct Flow {
        int32_t *d_tnb_off = nullptr;
        int32_t *d_tnb = nullptr;
        uint32_t *d_flow = nullptr;
        std::vector<std::pair<int64_t, int64_t>> groups;  // (first work entry, entries)
    } fl[4];
    uint64_t flow_launches = 0;

    static int slot(int b) { return b == 64 ? 0 : b == 128 ? 1 : b == 512 ? 3 : 2; }

    ~steps_batch() {
        for (auto &w : work) {
            if (w.graph) cudaGraphExecDestroy(w.graph);
            cudaFree(w.d);
        }
        for (auto &f : fl) {
            cudaFree(f.d_tnb_off);
            cudaFree(f.d_tnb);
            cudaFree(f.d_flow);
        }
        cudaFree(d_reps);
        cudaFree(d_err);
        cudaFreeHost(h_err);
        cudaFreeHost(h_last);
        cudaFreeHost(h_reps);
    }

    int build_work(int b) {
        Work &w = work[slot(b)];
        if (w.d) return STEPS_OK;
        std::vector<BlockWork> v;
        for (size_t j = 0; j < members.size(); ++j) {
            const int64_t tiles = (members[j]->T + b - 1) / b;
            for (int64_t t = 0; t < tiles; ++t) v.push_back(BlockWork{(int32_t)j, (int32_t)t});
        }
        w.n = (int64_t)v.size();
        if (w.n == 0) return STEPS_OK;
        if (!cuda_ok(cudaMalloc((void **)&w.d, v.size() * sizeof(BlockWork)), "steps_batch: alloc work"))
            return STEPS_ERR_OOM;
        if (!cuda_ok(cudaMemcpy(w.d, v.data(), v.size() * sizeof(BlockWork), cudaMemcpyHostToDevice),
                     "steps_batch: upload work"))
            return STEPS_ERR_CUDA;
        return STEPS_OK;
    }

    // the specialised batched kernel for block size b (compiled once); on
    // failure the generic kernel takes over unless specialisation was forced
    int prepare_spec(int b) {
        if (!use_spec || spec[slot(b)]) return STEPS_OK;
        spec[slot(b)] = spec_kernel(members[0]->model, b, &spec_why);
        if (spec[slot(b)]) return STEPS_OK;
        if (spec_forced) {
            set_error("steps_batch_run: the specialised batched kernel could not be built: " + spec_why);
            return STEPS_ERR_CUDA;
        }
        use_spec = false;
        return STEPS_OK;
    }

    int window(int b, cudaStream_t st) {  // one batched window + advance
        Work &w = work[slot(b)];
        int rc = use_spec && spec[slot(b)] ? launch_spec_batch(spec[slot(b)], w.d, w.n, d_reps, max_S, b, st)
                                           : launch_step_batch(w.d, w.n, d_reps, max_S, max_R, any_order0, b, st);
        if (!rc) rc = launch_advance(d_reps, (int32_t)members.size(), st);
        launches += 2;
        return rc;
    }

    int graph_for(int b) {
        Work &w = work[slot(b)];
        if (w.graph) return STEPS_OK;
        cudaStream_t cs = nullptr;
        if (!cuda_ok(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "cudaStreamCreate")) return STEPS_ERR_CUDA;
        cudaGraph_t g = nullptr;
        int rc = STEPS_OK;
        if (!cuda_ok(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture")) {
            cudaStreamDestroy(cs);
            return STEPS_ERR_CUDA;
        }
        const uint64_t before = launches;
        for (int q = 0; q < kGraphWindows && rc == STEPS_OK; ++q) rc = window(b, cs);
        launches = before;
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        if (rc == STEPS_OK && !cuda_ok(e, "cudaStreamEndCapture")) rc = STEPS_ERR_CUDA;
        if (rc == STEPS_OK && !cuda_ok(cudaGraphInstantiate(&w.graph, g, 0), "cudaGraphInstantiate")) rc = STEPS_ERR_CUDA;
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        return rc;
    }

    // the flow tables of block size b (once; build_work(b) first)
    int build_flow(int b) {
        Flow &f = fl[slot(b)];
        if (f.d_flow) return STEPS_OK;
        int dev = 0, l2 = 0;
        if (!cuda_ok(cudaGetDevice(&dev), "steps_batch: device") ||
            !cuda_ok(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev), "steps_batch: L2 size"))
            return STEPS_ERR_CUDA;
        std::vector<int32_t> off, nb, tmp;
        std::vector<std::pair<int64_t, int64_t>> groups;
        int64_t nwork = 0;
        try {
            int64_t gfirst = 0, gbytes = 0;
            for (steps_sim *m : members) {
                const int64_t B = b, T = m->T, tiles = (T + B - 1) / B, base = nwork;
                // counts (both buffers) and tables the member's windows touch
                const int64_t bytes = T * (8 * (int64_t)m->S + 40) + (m->d_rmask ? 4 * T : 0);
                if (nwork > gfirst && gbytes + bytes > (int64_t)l2 / 2) {
                    groups.emplace_back(gfirst, nwork - gfirst);
                    gfirst = nwork;
                    gbytes = 0;
                }
                gbytes += bytes;
                for (int64_t t = 0; t < tiles; ++t) {
                    tmp.assign(1, (int32_t)(base + t));
                    for (int64_t d = t * B; d < std::min(T, (t + 1) * B); ++d)
                        for (int q = 0; q < 4; ++q) {
                            const int32_t j = m->tab.nbr_dev[(size_t)(4 * d + q)];
                            if (j >= 0 && j / B != t) tmp.push_back((int32_t)(base + j / B));
                        }
                    std::sort(tmp.begin(), tmp.end());
                    tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
                    off.push_back((int32_t)nb.size());
                    nb.insert(nb.end(), tmp.begin(), tmp.end());
                }
                nwork += tiles;
            }
            off.push_back((int32_t)nb.size());
            if (nwork > gfirst) groups.emplace_back(gfirst, nwork - gfirst);
        } catch (const std::bad_alloc &) {
            set_error("steps_batch: flow tables: out of host memory");
            return STEPS_ERR_OOM;
        }
        if (nwork != work[slot(b)].n) {
            set_error("steps_batch: flow tables do not match the work list");
            return STEPS_ERR_STATE;
        }
        if (!cuda_ok(cudaMalloc((void **)&f.d_tnb_off, off.size() * 4), "steps_batch: flow tables") ||
            !cuda_ok(cudaMalloc((void **)&f.d_tnb, nb.size() * 4), "steps_batch: flow tables") ||
            !cuda_ok(cudaMalloc((void **)&f.d_flow, ((size_t)nwork + 1) * 4), "steps_batch: flow tables")) {
            cudaFree(f.d_tnb_off);
            cudaFree(f.d_tnb);
            cudaFree(f.d_flow);
            f.d_tnb_off = f.d_tnb = nullptr;
            f.d_flow = nullptr;
            return STEPS_ERR_OOM;
        }
        if (!cuda_ok(cudaMemcpy(f.d_tnb_off, off.data(), off.size() * 4, cudaMemcpyHostToDevice), "steps_batch") ||
            !cuda_ok(cudaMemcpy(f.d_tnb, nb.data(), nb.size() * 4, cudaMemcpyHostToDevice), "steps_batch") ||
            !cuda_ok(cudaMemset(f.d_flow, 0, ((size_t)nwork + 1) * 4), "steps_batch"))
            return STEPS_ERR_CUDA;
        f.groups = std::move(groups);
        return STEPS_OK;
    }

    // n full windows of every member as flow launches, one per group (the
    // device member table is not advanced: the table of any later window
    // is uploaded from the host)
    int flow_windows(int b, int64_t n) {
        int rc = build_flow(b);
        if (rc) return rc;
        Flow &f = fl[slot(b)];
        for (const auto &g : f.groups) {
            const int64_t cap = std::max<int64_t>(1, (int64_t)0x7FFFFFFF / g.second);
            for (int64_t done = 0; done < n;) {
                const int64_t nw = std::min(n - done, cap);
                if (!cuda_ok(cudaMemsetAsync(f.d_flow + work[slot(b)].n, 0, 4, stream), "steps_batch: flow counter"))
                    return STEPS_ERR_CUDA;
                FlowArgs a;
                a.tnb_off = f.d_tnb_off;
                a.tnb = f.d_tnb;
                a.tile_done = f.d_flow;
                a.fetch = f.d_flow + work[slot(b)].n;
                a.nwin = (uint32_t)nw;
                a.ntiles = (uint32_t)g.second;
                rc = launch_spec_batch_flow(spec[slot(b)], work[slot(b)].d, d_reps, a, (uint32_t)g.first, max_S, b,
                                            stream);
                if (rc) return rc;
                ++launches;
                ++flow_launches;
                done += nw;
            }
        }
        return STEPS_OK;
    }

    int run_windows(int b, int64_t n) {  // n windows at block size b
        int rc = build_work(b);
        if (!rc) rc = prepare_spec(b);
        if (rc) return rc;
        if (flow && use_spec && spec[slot(b)] && n >= 2) return flow_windows(b, n);
        int64_t done = 0;
        if (use_graph && n >= kGraphWindows) {
            rc = graph_for(b);
            if (rc) return rc;
            for (; n - done >= kGraphWindows; done += kGraphWindows) {
                if (!cuda_ok(cudaGraphLaunch(work[slot(b)].graph, stream), "cudaGraphLaunch")) return STEPS_ERR_CUDA;
                launches += 2 * kGraphWindows;
            }
        }
        for (; done < n; ++done) {
            rc = window(b, stream);
            if (rc) return rc;
        }
        return STEPS_OK;
    }
};

extern "C" {

void steps_batch_options_default(steps_batch_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->block = 0;
    opt->use_graph = 1;
}

int steps_batch_create(steps_sim *const *members, int32_t n, const steps_batch_options *opt, void *cuda_stream,
                       steps_batch **out) {
    CHECK_NULL(out, "steps_batch_create");
    *out = nullptr;
    CHECK_NULL(members, "steps_batch_create");
    if (n < 1) {
        set_error("steps_batch_create: need at least one member");
        return STEPS_ERR_ARG;
    }
    std::unique_ptr<steps_batch> b(new (std::nothrow) steps_batch);
    if (!b) return STEPS_ERR_OOM;
    steps_batch_options o;
    if (opt) o = *opt;
    else steps_batch_options_default(&o);
    if (o.block != 0 && o.block != 64 && o.block != 128 && o.block != 256 && o.block != 512) {
        set_error("steps_batch_create: block must be 0 (autotune), 64, 128, 256 or 512");
        return STEPS_ERR_ARG;
    }
    b->autotune = o.block == 0;
    b->block = o.block == 0 ? 256 : o.block;
    b->use_graph = o.use_graph != 0;
    if (o.flow != 0 && o.flow != 1) {
        set_error("steps_batch_create: flow must be 0 (window launches, default) or 1 (group flow launches)");
        return STEPS_ERR_ARG;
    }
    b->flow = o.flow == 1;
    b->stream = (cudaStream_t)cuda_stream;
    for (int32_t j = 0; j < n; ++j) {
        if (!members[j]) {
            set_error("steps_batch_create: NULL member");
            return STEPS_ERR_ARG;
        }
        for (int32_t q = 0; q < j; ++q)
            if (members[q] == members[j]) {
                set_error("steps_batch_create: a simulation appears twice");
                return STEPS_ERR_ARG;
            }
        b->members.push_back(members[j]);
        b->max_S = std::max(b->max_S, members[j]->S);
        b->max_R = std::max(b->max_R, members[j]->model.R);
        b->any_order0 = b->any_order0 || members[j]->model.dev.order0 != 0u;
    }
    if (!cuda_ok(cudaMallocHost((void **)&b->h_reps, sizeof(RepEntry) * n), "steps_batch_create: host alloc") ||
        !cuda_ok(cudaMallocHost((void **)&b->h_last, sizeof(RepEntry) * n), "steps_batch_create: host alloc") ||
        !cuda_ok(cudaMallocHost((void **)&b->h_err, 4), "steps_batch_create: host alloc") ||
        !cuda_ok(cudaMalloc((void **)&b->d_reps, sizeof(RepEntry) * n), "steps_batch_create: alloc") ||
        !cuda_ok(cudaMalloc((void **)&b->d_err, 4), "steps_batch_create: alloc") ||
        !cuda_ok(cudaMemset(b->d_err, 0, 4), "steps_batch_create: memset"))
        return STEPS_ERR_OOM;
    // the model-specialised batched kernel: all members must share one model structure
    bool uniform = true;
    int64_t tets = 0;
    const std::string src0 = spec_program_source(members[0]->model, 256);
    for (int32_t j = 0; j < n; ++j) {
        tets += members[j]->T;
        if (j > 0 && uniform && spec_program_source(members[j]->model, 256) != src0) uniform = false;
    }
    if (o.specialize > 0 && !uniform) {
        set_error("steps_batch_create: specialize = 1 needs members that share one model structure");
        return STEPS_ERR_ARG;
    }
    constexpr int64_t kSpecializeMinTets = 65536;
    bool any_exp = false;
    for (int32_t j = 0; j < n; ++j) any_exp = any_exp || members[j]->model.leave_exp;
    if (any_exp && (!uniform || o.specialize < 0)) {
        set_error("steps_batch_create: members with the EXP leave law run on the model-specialised batched "
                  "kernel only: they need one model structure and specialize 0 or 1");
        return STEPS_ERR_ARG;
    }
    b->spec_forced = o.specialize > 0 || any_exp;
    b->use_spec = uniform && (o.specialize > 0 || any_exp || (o.specialize == 0 && tets >= kSpecializeMinTets));
    if (b->use_spec)
        for (steps_sim *m : b->members) {
            int rc = m->ensure_trial();
            if (rc) return rc;
        }
    int rc = b->build_work(b->block);
    if (rc) return rc;
    *out = b.release();
    return STEPS_OK;
}

void steps_batch_destroy(steps_batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    delete b;
}

}  // extern "C"

namespace steps {

// steps_batch_run without its final wait: every window is enqueued on the
// batch's stream, the members' clocks advanced and the error word's copy to
// the host enqueued. batch_finish waits and turns the word into a code.
int batch_enqueue(steps_batch *b, const double *t_end) {
    CHECK_NULL(b, "steps_batch_run");
    CHECK_NULL(t_end, "steps_batch_run");
    const size_t n = b->members.size();
    for (size_t j = 0; j < n; ++j)
        if (!std::isfinite(t_end[j])) {
            set_error("steps_batch_run: t_end must be finite");
            return STEPS_ERR_ARG;
        }
    for (steps_sim *m : b->members)
        if (int rf = refuse_failed(m, "steps_batch_run")) return rf;
    // members' own streams may still hold work
    for (steps_sim *m : b->members)
        if (!cuda_ok(cudaStreamSynchronize(m->stream), "steps_batch_run: member stream")) return STEPS_ERR_CUDA;
    // the window schedule of every member (the loop of steps_run)
    std::vector<int64_t> nfull(n, 0);
    std::vector<double> partial(n, 0.0);  // > 0: a shortened last window of this length
    int64_t nmax = 0;
    for (size_t j = 0; j < n; ++j) {
        steps_sim *m = b->members[j];
        const double tau = m->tab.tau;
        const bool finite = std::isfinite(tau);
        const double tol = finite ? 1e-9 * tau : 0.0;
        int64_t k = 0;
        for (;;) {
            const int64_t kk = m->k_grid + k;
            const double t = kk == 0 ? m->t_base : m->t_base + (double)kk * tau;
            if (!(t_end[j] - t > tol)) break;
            if (finite && t + tau <= t_end[j] + tol) {
                ++k;
            } else {
                partial[j] = t_end[j] - t;
                break;
            }
        }
        nfull[j] = k;
        nmax = std::max(nmax, k);
    }
    // table for the full windows
    for (size_t j = 0; j < n; ++j) {
        steps_sim *m = b->members[j];
        RepEntry &e = b->h_reps[j];
        std::memset(&e, 0, sizeof(e));
        e.model = m->model.dev;
        e.args = m->args(0, m->k_total, nullptr, std::isfinite(m->tab.tau) ? m->tab.tau : 1.0, m->scale_full);
        e.args.err = b->d_err;
        e.cnt[0] = m->d_cnt[0];
        e.cnt[1] = m->d_cnt[1];
        e.parity = (uint32_t)m->cur;
        e.window_end = m->k_total + (uint64_t)nfull[j];
    }
    if (!cuda_ok(cudaMemcpyAsync(b->d_reps, b->h_reps, sizeof(RepEntry) * n, cudaMemcpyHostToDevice, b->stream),
                 "steps_batch_run: upload"))
        return STEPS_ERR_CUDA;
    int64_t done = 0;
    int rc = STEPS_OK;
    if (b->autotune && nmax >= 12) {
        // time the candidate block sizes on alternating windows (one warm window
        // each, then two rounds of one timed window each), so that the state's
        // slow drift over the run cancels; keep 256 unless another is more than
        // 2 % faster
        const int cand[3] = {128, 256, 512};
        b->tune_ms.assign(3, 0.f);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (!cuda_ok(cudaEventCreate(&e0), "steps_batch_run: autotuner event") ||
            !cuda_ok(cudaEventCreate(&e1), "steps_batch_run: autotuner event")) {
            if (e0) cudaEventDestroy(e0);
            return STEPS_ERR_CUDA;
        }
        float total[3] = {0.f, 0.f, 0.f};
        for (int round = 0; round < 2 && rc == STEPS_OK; ++round) {
            for (int c = 0; c < 3 && rc == STEPS_OK; ++c) {
                rc = b->build_work(cand[c]);
                if (rc) break;
                if (round == 0) {
                    rc = b->run_windows(cand[c], 1);  // warm
                    if (rc) break;
                    done += 1;
                }
                float ms = 0.f;
                if (!cuda_ok(cudaEventRecord(e0, b->stream), "steps_batch_run: autotuner") ||
                    (rc = b->run_windows(cand[c], 1)) != STEPS_OK ||
                    !cuda_ok(cudaEventRecord(e1, b->stream), "steps_batch_run: autotuner") ||
                    !cuda_ok(cudaEventSynchronize(e1), "steps_batch_run: autotuner") ||
                    !cuda_ok(cudaEventElapsedTime(&ms, e0, e1), "steps_batch_run: autotuner")) {
                    if (rc == STEPS_OK) rc = STEPS_ERR_CUDA;
                    break;
                }
                total[c] += ms;
                done += 1;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc) return rc;
        int best_b = 256;
        float best = total[1];
        for (int c = 0; c < 3; ++c) {
            b->tune_ms[c] = total[c] / 2.f;
            if (total[c] < 0.98f * best) {
                best = total[c];
                best_b = cand[c];
            }
        }
        b->block = best_b;
        b->autotune = false;
    }
    rc = b->run_windows(b->block, nmax - done);
    if (rc) return rc;
    // shortened last windows: their table goes into the second pinned buffer
    // (h_reps may still be read by its queued upload)
    bool any_partial = false;
    for (size_t j = 0; j < n; ++j) {
        steps_sim *m = b->members[j];
        RepEntry &e = b->h_last[j];
        e = b->h_reps[j];
        const uint64_t w = m->k_total + (uint64_t)nfull[j];
        e.args.window = w;
        e.parity = (uint32_t)(m->cur ^ (int)(nfull[j] & 1));
        e.window_end = w;
        if (partial[j] > 0.0) {
            any_partial = true;
            uint32_t scale[kMaxSpecies] = {};
            for (int s = 0; s < m->S; ++s) scale[s] = species_scale(m->model, m->tab, s, partial[j]);
            if (partial[j] != m->tab.tau) {
                int rl = m->upload_leave(partial[j], b->stream);  // after the full windows, in stream order
                if (rl) return rl;
            }
            StepArgs a = m->args(0, w, nullptr, partial[j], scale);
            a.err = b->d_err;
            e.args = a;
            e.window_end = w + 1;
        }
    }
    if (any_partial) {
        if (!cuda_ok(cudaMemcpyAsync(b->d_reps, b->h_last, sizeof(RepEntry) * n, cudaMemcpyHostToDevice, b->stream),
                     "steps_batch_run: upload"))
            return STEPS_ERR_CUDA;
        rc = b->run_windows(b->block, 1);
        if (rc) return rc;
    }
    // members' clocks and buffers
    for (size_t j = 0; j < n; ++j) {
        steps_sim *m = b->members[j];
        const int64_t wins = nfull[j] + (partial[j] > 0.0 ? 1 : 0);
        m->k_total += (uint64_t)wins;
        m->launches += (uint64_t)wins;
        m->cur ^= (int)(wins & 1);
        if (partial[j] > 0.0) {
            m->t_base = t_end[j];
            m->k_grid = 0;
        } else {
            m->k_grid += nfull[j];
        }
    }
    if (!cuda_ok(cudaMemcpyAsync(b->h_err, b->d_err, 4, cudaMemcpyDeviceToHost, b->stream),
                 "steps_batch_run: error word"))
        return STEPS_ERR_CUDA;
    return STEPS_OK;
}

int batch_finish(steps_batch *b) {
    if (!cuda_ok(cudaStreamSynchronize(b->stream), "steps_batch_run")) return STEPS_ERR_CUDA;
    const uint32_t err = *b->h_err;
    if (err) {
        cudaMemset(b->d_err, 0, 4);
        if (err & 4u) {
            for (steps_sim *m : b->members) m->failed = true;
            set_error("steps_batch_run: a bulk copy into shared memory did not complete within its wait limit; "
                      "a copy may still be in flight, so every member is closed to further runs");
            return STEPS_ERR_TIMEOUT;
        }
        set_error(err & 2u ? "steps_batch_run: a tet fired more than 2^24 reactions in one window"
                           : "steps_batch_run: a negative count was seen on the device");
        return STEPS_ERR_STATE;
    }
    return STEPS_OK;
}

std::string sim_structure_key(const steps_sim *sim) { return spec_program_source(sim->model, 256); }

}  // namespace steps

extern "C" {

int steps_batch_run(steps_batch *b, const double *t_end) {
    int rc = steps::batch_enqueue(b, t_end);
    return rc ? rc : steps::batch_finish(b);
}

int steps_batch_specialized(const steps_batch *b, int32_t *specialized) {
    CHECK_NULL(b, "steps_batch_specialized");
    CHECK_NULL(specialized, "steps_batch_specialized");
    *specialized = b->use_spec ? 1 : 0;
    return STEPS_OK;
}

int steps_batch_info(const steps_batch *b, int32_t *block, uint64_t *launches, float *tune_ms) {
    CHECK_NULL(b, "steps_batch_info");
    if (block) *block = b->block;
    if (launches) *launches = b->launches;
    if (tune_ms)
        for (int c = 0; c < 3; ++c) tune_ms[c] = c < (int)b->tune_ms.size() ? b->tune_ms[c] : 0.f;
    return STEPS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free run on caller-owned device counts.
//
// Scratch for steps_run_noalloc lives in this file-scope device array: two
// receiving/sending count buffers of up to kNoAllocMaxCounts int32 each, then
// an error word. Every GPU that loads the library holds it (32 MiB + 256 B)
// until the process exits. Host code cannot use the array's name as a device
// address; the address is looked up once per device with
// cudaGetSymbolAddress, with that device current.
// ---------------------------------------------------------------------------
constexpr size_t kNoAllocMaxCounts = (size_t)1 << 22;  // n_species * Tpad per buffer
static __device__ __align__(256) int32_t g_noalloc_scratch[2 * kNoAllocMaxCounts + 64];

namespace {

struct NoAllocScratch {
    bool ready = false;
    int32_t *counts = nullptr;  // [2][kNoAllocMaxCounts]
    uint32_t *err = nullptr;    // two words after the count buffers: window error word, input check flag
};

constexpr int kNoAllocMaxDevices = 64;
NoAllocScratch g_noalloc_dev[kNoAllocMaxDevices];
std::mutex g_noalloc_mu;

int noalloc_scratch(NoAllocScratch &out) {
    int dev = -1;
    if (!cuda_ok(cudaGetDevice(&dev), "steps_run_noalloc: cudaGetDevice")) return STEPS_ERR_CUDA;
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("steps_run_noalloc: device index out of range");
        return STEPS_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocScratch &s = g_noalloc_dev[dev];
    if (!s.ready) {
        void *p = nullptr;
        if (!cuda_ok(cudaGetSymbolAddress(&p, g_noalloc_scratch), "steps_run_noalloc: cudaGetSymbolAddress"))
            return STEPS_ERR_CUDA;
        s.counts = static_cast<int32_t *>(p);
        s.err = reinterpret_cast<uint32_t *>(s.counts + 2 * kNoAllocMaxCounts);
        s.ready = true;
    }
    out = s;
    return STEPS_OK;
}

}  // namespace

extern "C" int steps_run_noalloc(steps_sim *sim, int32_t *d_counts, double t_end) {
    CHECK_NULL(sim, "steps_run_noalloc");
    CHECK_NULL(d_counts, "steps_run_noalloc");
    if (!std::isfinite(t_end)) {
        set_error("steps_run_noalloc: t_end must be finite");
        return STEPS_ERR_ARG;
    }
    const size_t S = (size_t)sim->S, T = (size_t)sim->T, Tpad = (size_t)sim->Tpad;
    if (S * Tpad > kNoAllocMaxCounts) {
        set_error("steps_run_noalloc: n_species * padded tets = " + std::to_string(S * Tpad) +
                  " exceeds the fixed scratch of " + std::to_string(kNoAllocMaxCounts) +
                  " counts; use steps_run");
        return STEPS_ERR_ARG;
    }
    if (int rf = refuse_failed(sim, "steps_run_noalloc")) return rf;
    if (sim->d_leave[0]) {
        set_error("steps_run_noalloc: the EXP leave law needs a host-built table for a shortened window; "
                  "use steps_run");
        return STEPS_ERR_ARG;
    }
    // the scratch address is per device, and the simulation's stream and
    // tables belong to the device it was created on
    int dev = -1;
    if (!cuda_ok(cudaGetDevice(&dev), "steps_run_noalloc: cudaGetDevice")) return STEPS_ERR_CUDA;
    if (dev != sim->device) {
        set_error("steps_run_noalloc: the current device (" + std::to_string(dev) +
                  ") is not the one the simulation was created on (" + std::to_string(sim->device) +
                  "); make that device current first");
        return STEPS_ERR_ARG;
    }
    NoAllocScratch sc;
    int rc = noalloc_scratch(sc);
    if (rc) return rc;
    int32_t *buf[2] = {sc.counts, sc.counts + kNoAllocMaxCounts};
    cudaStream_t st = sim->stream;
    // the scratch keeps the previous call's contents: clear both buffers
    // (padding and receiving rows must be zero) and both error words
    if (!cuda_ok(cudaMemsetAsync(buf[0], 0, S * Tpad * 4, st), "steps_run_noalloc: clear") ||
        !cuda_ok(cudaMemsetAsync(buf[1], 0, S * Tpad * 4, st), "steps_run_noalloc: clear") ||
        !cuda_ok(cudaMemsetAsync(sc.err, 0, 8, st), "steps_run_noalloc: clear"))
        return STEPS_ERR_CUDA;
    // reject negative input counts before anything (clock, caller's buffer) changes
    {
        const int64_t n = (int64_t)(S * T);
        uint32_t neg = 0;
        any_negative<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(d_counts, n, sc.err + 1);
        if (!cuda_ok(cudaGetLastError(), "steps_run_noalloc: check") ||
            !cuda_ok(cudaMemcpyAsync(&neg, sc.err + 1, 4, cudaMemcpyDeviceToHost, st), "steps_run_noalloc: check") ||
            !cuda_ok(cudaStreamSynchronize(st), "steps_run_noalloc: check"))
            return STEPS_ERR_CUDA;
        if (neg) {
            set_error("steps_run_noalloc: negative count in d_counts");
            return STEPS_ERR_ARG;
        }
    }
    const unsigned grid = (unsigned)((T + 255) / 256);
    scatter_to_device_order<<<grid, 256, 0, st>>>(d_counts, (int64_t)T, (int32_t)S, sim->d_inv_perm, buf[0], Tpad);
    if (!cuda_ok(cudaGetLastError(), "steps_run_noalloc: scatter")) return STEPS_ERR_CUDA;

    // the window loop of steps_run (Algorithm 1), with plain launches on the scratch buffers
    const double tau = sim->tab.tau;
    const bool finite = std::isfinite(tau);
    const double tol = finite ? 1e-9 * tau : 0.0;
    int cur = 0;
    auto launch = [&](double tau_k, const uint32_t *scale) -> int {
        StepArgs a = sim->args(0, sim->k_total, nullptr, tau_k, scale);
        a.cur = buf[cur];
        a.nxt = buf[1 - cur];
        a.err = sc.err;
        int r = sim->launch(a, st);
        if (r) return r;
        ++sim->launches;
        ++sim->k_total;
        cur = 1 - cur;
        return STEPS_OK;
    };
    for (;;) {
        const double t = sim->time();
        if (!(t_end - t > tol)) break;
        if (finite && t + tau <= t_end + tol) {
            rc = launch(tau, sim->scale_full);
            if (rc) return rc;
            sim->k_grid += 1;
        } else {
            uint32_t scale[kMaxSpecies] = {};
            for (int s = 0; s < sim->S; ++s) scale[s] = species_scale(sim->model, sim->tab, s, t_end - t);
            rc = launch(t_end - t, scale);
            if (rc) return rc;
            sim->t_base = t_end;
            sim->k_grid = 0;
            break;
        }
    }
    gather_to_original_order<<<grid, 256, 0, st>>>(buf[cur], (int64_t)T, (int32_t)S, sim->d_inv_perm, Tpad, d_counts);
    if (!cuda_ok(cudaGetLastError(), "steps_run_noalloc: gather")) return STEPS_ERR_CUDA;
    uint32_t err = 0;
    if (!cuda_ok(cudaMemcpyAsync(&err, sc.err, 4, cudaMemcpyDeviceToHost, st), "steps_run_noalloc: error word") ||
        !cuda_ok(cudaStreamSynchronize(st), "steps_run_noalloc"))
        return STEPS_ERR_CUDA;
    if (err & 4u) {
        sim->failed = true;
        set_error("steps_run_noalloc: a bulk copy into shared memory did not complete within its wait limit; "
                  "a copy may still be in flight, so this simulation is closed to further runs");
        return STEPS_ERR_TIMEOUT;
    }
    if (err) {
        set_error(err & 2u ? "steps_run_noalloc: a tet fired more than 2^24 reactions in one window"
                           : "steps_run_noalloc: a negative count was seen on the device");
        return STEPS_ERR_STATE;
    }
    return STEPS_OK;
}
