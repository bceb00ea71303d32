// Declarations the device code needs: model and window argument layouts and
// the constants of the step. Includes nothing from the C++ standard library,
// so that the run-time compiler (NVRTC) can build model-specialised kernels
// from the same sources.
#pragma once

#ifdef __CUDACC_RTC__
typedef signed char int8_t;
typedef unsigned char uint8_t;
typedef short int16_t;
typedef unsigned short uint16_t;
typedef int int32_t;
typedef unsigned int uint32_t;
typedef long long int64_t;
typedef unsigned long long uint64_t;
#else
#include <cstddef>
#include <cstdint>
#include <vector_types.h>
#endif

namespace steps {

constexpr int kMaxSpecies = 32;  // STEPS_MAX_SPECIES
constexpr int kMaxReac = 32;     // STEPS_MAX_REACTIONS
constexpr int kMaxChanges = 6;
constexpr double kAvogadro = 6.02214076e23;
// Reaction events one tet may fire in one window before the kernel gives up
// on it and raises error bit 2 (a guard against runaway rate constants).
constexpr uint32_t kMaxEventsPerWindow = 1u << 24;
// Full windows counted and enqueued per batch by steps_run.
constexpr int64_t kWindowBatch = 1 << 16;

// Stream purposes of the counter-based generator (top 4 bits of counter word 3).
constexpr uint32_t kPurposeReac = 1;
constexpr uint32_t kPurposeRound = 2;
constexpr uint32_t kPurposeDiff = 3;
constexpr uint32_t kPurposeBulk = 4;  // bit planes of species with many trial molecules in a tet
// trial molecules of a species in a tet from which it draws by bit planes
constexpr int32_t kBulkMin = 16;

// Reaction kinds by propensity form.
enum ReacType : int8_t { kOrder0 = 0, kOrder1 = 1, kOrder2 = 2, kDimer = 3 };

// ---------------------------------------------------------------- device-side model
// Propensity a = ((c x) y) in float with x = count of species ia, y = count
// of species ib minus sub; row S of the kernel's count tile holds 1, so a
// missing reactant reads 1. c = k (order 1), k / (N_A V) (order 2 and dimer:
// y = n - 1) or k N_A V (order 0), the last two computed per tet.
struct ReacDesc {
    float k;                      // rate constant, float
    uint32_t need;                // bit s set when species s is a reactant (a_r = 0 unless all are present)
    int32_t ia, ib;               // count rows read for x and y (S = the row of ones)
    int32_t sub;                  // subtracted from y: 1 for a dimer, else 0
    int32_t type;                 // ReacType
    int32_t nchg;                 // species changed (delta != 0), increasing species order
    int8_t chg_s[kMaxChanges];
    int8_t chg_d[kMaxChanges];
};

struct ModelDev {
    int32_t S, R;
    uint32_t diffusive;           // bit s set when D_s > 0
    uint32_t order0;              // bit r set when reaction r has order 0
    ReacDesc reac[kMaxReac];
};

// Arguments of one diffusion window.
struct StepArgs {
    int32_t *cur;                 // [S][Tpad] counts at window start; non-zero entries are zeroed as read
    int32_t *nxt;                 // [S][Tpad] counts at window end (all entries must be zero on entry)
    const int4 *nbr;              // [T] face neighbours (device index), -1 = boundary
    const uint4 *thr;             // [T] cumulative face thresholds at the full window, 2^31 fixed point
    const float *inv_nav;         // [T] 1 / (N_A V_L) as float
    const int32_t *orig;          // [T] original tet id (RNG key), or nullptr for identity
    const uint32_t *rmask;        // [T] active-reaction bits, or nullptr = all active
    uint32_t *err;                // device error word
    int32_t T, Tpad;
    uint32_t key0, key1;          // Philox key = seed
    uint64_t window;              // window index of this launch (RNG counter)
    const uint64_t *window_base;  // if set, window = *window_base + window (graph replay)
    double tau_k, inv_tau_k;
    float tau_dn;                 // largest float <= tau_k
    int32_t occ;                  // STEPS_OCC_*
    int32_t prefetch;             // tiles ahead whose tables a block prefetches into L2 (0 = none)
    int32_t *trial;               // [S][Tpad] trial counts, for kernels that keep them in global memory
    const uint32_t *leave;        // [S][Tpad] EXP leave law: floor(2^31 (1 - exp(-tau_k D_S G_tet))), or nullptr
    uint32_t scale[kMaxSpecies];  // per-species fixed-point scale for this window length
};

// Full windows of one simulation in one flow launch (flow_tiles; the batched
// form: a group of members, batch_flow_tile): one block per item (window q,
// tile t), q-major; the item (q, t) waits until every tile sharing a face
// with t, t included, has finished window q - 1.
struct FlowArgs {
    const int32_t *tnb_off;  // [ntiles + 1] offsets into tnb of each tile's neighbour tiles
    const int32_t *tnb;      // neighbour tiles (each tile lists itself)
    uint32_t *tile_done;     // [ntiles] low word of (last window the tile finished + 1)
    uint32_t *fetch;         // item counter, zero when the launch starts
    uint32_t nwin;           // windows a.window, a.window + 1, ... (nwin * ntiles < 2^31)
    uint32_t ntiles;
};

// One member of a batched launch, resident in device memory. The step kernel
// reads its member's model and arguments from here (cur/nxt chosen by
// `parity`); the advance kernel moves `args.window` and `parity` after every
// window while args.window < window_end.
struct RepEntry {
    ModelDev model;
    StepArgs args;
    int32_t *cnt[2];
    uint32_t parity;
    uint32_t pad_;
    uint64_t window_end;
};

// A block of a batched launch: member index and tile (BLOCK consecutive tets) within it.
struct BlockWork {
    int32_t rep;
    int32_t tile;
};

}  // namespace steps
