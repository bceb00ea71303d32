// Internal declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <vector_types.h>

#include "../../include/steps_gpu.h"
#include "steps_device.h"

namespace steps {

static_assert(kMaxSpecies == STEPS_MAX_SPECIES && kMaxReac == STEPS_MAX_REACTIONS, "limits");

void set_error(const std::string &msg);

// ---------------------------------------------------------------- host objects
struct HostMesh {
    int64_t nv = 0, nt = 0;
    std::vector<double> verts;    // [nv*3]
    std::vector<int32_t> tets;    // [nt*4]
    std::vector<int32_t> nbr;     // [nt*4] original order, -1 boundary
    std::vector<double> vol;      // [nt] m^3
    std::vector<double> g;        // [nt*4] A/(V d), 0 on boundary
    std::vector<double> bary;     // [nt*3]
};

struct HostModel {
    int32_t S = 0, R = 0;
    std::vector<double> D;        // [S]
    std::vector<int32_t> lhs, rhs;  // [R*S]
    std::vector<double> k;        // [R]
    ModelDev dev{};
    bool leave_exp = false;       // the simulation's leave law is EXP (p = 1 - exp(-tau d))
};

// steps_host.cpp
int build_mesh(const double *verts, int64_t nv, const int32_t *tets, int64_t nt, HostMesh &m);
int build_model(int32_t S, const double *D, int32_t R, const int32_t *lhs, const int32_t *rhs,
                const double *k, HostModel &m);

struct Tables {
    double tau = 0, dmax = 0, gmax = 0;
    std::vector<int32_t> perm;      // device index -> original id
    std::vector<int32_t> inv_perm;  // original id -> device index
    std::vector<int32_t> nbr_dev;   // [T*4] device order, device indices
    std::vector<uint32_t> thr_dev;  // [T*4] device order
    std::vector<float> inv_nav_dev; // [T]
    std::vector<double> G_dev;      // [T] device order: sum of the face rates g over internal faces
};
void build_tables(const HostMesh &mesh, const HostModel &model, int reorder, Tables &t);
uint32_t species_scale(const HostModel &model, const Tables &t, int s, double tau_k);
// EXP leave law: out[s * Tpad + d] = floor(2^31 (1 - exp(-(tau_k D_s) G_d))) for every
// species and device-order tet (0 for immobile species and the padding).
void exp_leave_table(const HostModel &model, const Tables &t, double tau_k, size_t Tpad, std::vector<uint32_t> &out);

// steps_kernels.cu
// L2 prefetch distance in tiles: half of the blocks of a kernel resident on
// the whole GPU at once (SMs x blocks per SM), cached per kernel and
// shared-memory size.
int prefetch_distance(const void *kernel, int block, size_t smem);
int launch_step(const ModelDev &m, const StepArgs &a, int block, void *stream);
int launch_philox_test(uint64_t seed, const uint32_t *d_ctr, int64_t n, uint32_t *d_out, void *stream);
int launch_logf_test(const float *d_x, int64_t n, float *d_out, void *stream);
int launch_wait_test(const void *d_src, int deliver, long long limit, uint32_t *d_status, void *stream);
int launch_flow_wait_test(const int32_t *d_off, const int32_t *d_nb, uint32_t *d_done, long long limit,
                          uint32_t *d_status);
int launch_add_u64(uint64_t *p, uint64_t v, void *stream);
int launch_step_batch(const BlockWork *work, int64_t nblocks, RepEntry *reps, int max_S, int max_R,
                      bool any_order0, int block, void *stream);
int launch_advance(RepEntry *reps, int32_t n, void *stream);

// steps_spec.cpp: the plain and batched step kernels specialised for one
// model by the run-time compiler (an opaque handle, cached process-wide);
// nullptr (with the reason in *why) when they cannot be built.
void *spec_kernel(const HostModel &hm, int block, std::string *why);
int launch_spec(void *spec, const ModelDev &m, const StepArgs &a, int block, void *stream);
// Full windows a.window .. a.window + f.nwin - 1 in one launch of the flow
// kernel (one block per item: f.nwin x f.ntiles blocks); f.fetch must be zero.
int launch_spec_flow(void *spec, const ModelDev &m, const StepArgs &a, const FlowArgs &f, int block, void *stream);
// The same on the generic step kernel (block must be 256).
int launch_flow(const ModelDev &m, const StepArgs &a, const FlowArgs &f, int block, void *stream);
// Full windows of the batch members whose tiles are work[work0 .. work0 + f.ntiles) in one launch of
// the batched flow kernel (f.nwin windows from each member's current window); f.fetch must be zero.
int launch_spec_batch_flow(void *spec, const BlockWork *work, RepEntry *reps, const FlowArgs &f, uint32_t work0, int S,
                           int block, void *stream);
int launch_spec_batch(void *spec, const BlockWork *work, int64_t nblocks, RepEntry *reps, int S, int block,
                      void *stream);
std::string spec_program_source(const HostModel &hm, int block);
// whether the specialised kernels keep the trial counts in StepArgs::trial
bool spec_global_trial(const HostModel &hm);

// steps_api.cu: steps_batch_run in two parts (enqueue every window and the
// error word's copy; then wait and map the word to a return code), so that
// batches on different streams can run at the same time; and a key that is
// equal for simulations whose models share one structure (one specialised
// kernel serves them all).
int batch_enqueue(steps_batch *b, const double *t_end);
int batch_finish(steps_batch *b);
std::string sim_structure_key(const steps_sim *sim);

}  // namespace steps
