// Internal interface between the C ABI (ea_api.cu) and the kernels (ea_kernels.cu).
//
// Device layout of one ensemble:
//   spins  [G][C][NT][2][H]   colour-split: word (colour, k) holds site 2k + (x parity),
//                             k = i >> 1, H = N / 2; unit (g, c) owns NT*N contiguous words
//   bonds  [G][3][2][H]       bond words in the same colour-split order
//   energy [G][C][NT][32]     int32 energies by slot
// The colour-split order makes the four sites of one Philox call (class
// indices 4q..4q+3 of one colour) one aligned 16-byte vector.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ea.h"

namespace ea {

constexpr int kLanes = 32;
constexpr int kMaxTemps = 64;
constexpr int kPlanes = 8;          // bit planes of a thread's energy counter (sum <= 255)
constexpr int kMaxQuadsPerThread = 10;  // 4 sites x 6 bonds x 10 quads = 240 <= 255
constexpr int kMaxThreads = 512;        // per CTA of the sweep kernels (128 registers a thread)

struct RoundKeys {
    uint32_t k[20];                 // Philox key of rounds 0..9: (k0 + r*W0, k1 + r*W1)
};

RoundKeys make_round_keys(uint64_t seed);

// Everything one sweep launch needs.  Pointers are device pointers.
struct SweepLaunch {
    uint32_t *spins;
    const uint32_t *bonds;
    const uint32_t *metro;          // [NT][3]
    const uint32_t *swapt;          // [NT-1][swap_len]
    uint32_t swap_len;
    int32_t *energy;                // [G][C][NT][32]
    uint32_t G, NT, C;
    RoundKeys rk;
    uint64_t s0;                    // global index of the first sweep
    uint32_t n_sweeps;
    uint32_t swap_every;
    uint64_t P0;                    // global index of the first swap pass of this launch
    uint32_t pass_local0;           // index into swap_log of that pass
    int32_t *energy_log;            // [n_log][G][NT][C][32], row = s - log_s0
    uint64_t log_s0;
    uint32_t *swap_log;             // [passes][G][C][NT-1]
    uint64_t *qhist;                // [NT][N+1]
    int64_t *esum;                  // [NT]
    uint64_t measure_from;
    uint32_t measure_every;
    int *err;
    // chunked form: lattices [t0, t0 + nlat) of each unit per CTA
    uint32_t t_per_cta;
    int compute_energy_last;        // chunked form: energies after the last sweep
    // external field h = h_num / h_den (h_num == 0: none); see ea_device.cuh
    const uint64_t *metro_f;        // [NT][2][7] thresholds, 2^32 = always
    int32_t *mag;                   // [G][C][NT][32] magnetisations by slot
    int32_t h_num, h_den, step;     // step of Et = h_den E - h_num M differences
    uint32_t g_base;                // global index of word-group 0 in the random-number counters
};

enum PlanForm { kFormUnit = 0, kFormUnitFast = 1, kFormChunked = 2, kFormUnitWave = 3 };

struct Plan {
    int form;               // PlanForm
    bool unit;              // all NT lattices of a (g, c) unit in one CTA (swaps in-kernel)
    int threads_per_lattice;    // generic forms: threads per lattice; fast form: threads per
                                // (lattice, row parity) class
    int lattices_per_cta;   // == NT for the unit forms
    int threads;
    size_t smem;
    bool j_in_smem;
    bool swap_in_smem;      // unit forms: swap threshold table staged in shared memory
    int field_kind = 0;     // wavefront form in a field: 34 or 43 (wave_field_kind), else 0
};

bool supported_L(int L);
// Every kernel plan that can run (L, NT) within the device's opt-in shared
// memory, best guess first.  Empty if none.
// field: plans for the external-field kernels (generic unit and chunked forms).
// field_kind: the wavefront kernel's field kind for this field (0: the field
// runs the generic forms only).
std::vector<Plan> make_plans(int L, int NT, int C, uint32_t swap_len, size_t smem_optin,
                             bool field = false, int field_kind = 0);

int fast_unit_threads(int L, int HP, int NT);
// Unit kernel with the wavefront replica exchange (L = 8, NT <= kWaveMaxTemps,
// one warp per two slots; launches without qhist / esum measurement).
// In an external field the kernel takes the fields whose always-accept
// boundaries are u >= 3 for one spin value and u >= 4 for the other
// (wave_field_kind: 34 or 43; 0 for any other pair).
constexpr int kWaveMaxTemps = 32;
int wave_unit_threads(int L, int NT);
size_t wave_unit_smem(int L, int NT, uint32_t swap_len, bool swap_smem, bool field = false,
                      bool overlaps = false);
int wave_field_kind(int ua0, int ua1);
// meas: 0 none; 1 energy sums (esum); 2 energy sums and the q histogram (C = 2)
cudaError_t launch_sweep_unit_wave(const SweepLaunch &a, bool swap_in_smem, int field_kind, int meas,
                                   cudaStream_t st, uint64_t *launches);
// Dynamic shared memory of the specialised unit kernel (with or without the
// swap table, the measurement snapshots and the shared-memory histogram).
size_t fast_unit_smem(int L, int NT, uint32_t swap_len, bool swap_smem, bool snap, bool hist_smem);
cudaError_t launch_sweep_unit_fast(const SweepLaunch &a, int L, int HP, bool swap_in_smem,
                                   bool cluster_measure, size_t smem_optin, cudaStream_t st,
                                   uint64_t *launches);

// Launchers: return cudaSuccess or the launch error.  Each adds its kernel
// count to *launches.
cudaError_t launch_import(const uint32_t *api_spins, const uint32_t *api_bonds, uint32_t *spins,
                          uint32_t *bonds, int L, uint32_t G, uint32_t NT, uint32_t C,
                          cudaStream_t st, uint64_t *launches);
cudaError_t launch_export(const uint32_t *spins, uint32_t *api_spins, int L, uint32_t G,
                          uint32_t NT, uint32_t C, cudaStream_t st, uint64_t *launches);
cudaError_t launch_import_spins(const uint32_t *api_spins, uint32_t *spins, int L, uint32_t G,
                                uint32_t NT, uint32_t C, cudaStream_t st, uint64_t *launches);
cudaError_t launch_sweep_unit(const SweepLaunch &a, int L, const Plan &plan, bool cluster_measure,
                              cudaStream_t st, uint64_t *launches);
cudaError_t launch_sweep_chunk(const SweepLaunch &a, int L, const Plan &plan, cudaStream_t st,
                               uint64_t *launches);
cudaError_t launch_swap_global(const SweepLaunch &a, int L, uint64_t P, uint32_t *masks,
                               int32_t *energy_log_row, cudaStream_t st, uint64_t *launches);
// Per-plane counts (k_measure_planes); L <= 32.
cudaError_t launch_measure_planes(const uint32_t *spins, int L, uint32_t G, uint32_t NT, uint32_t C,
                                  int mode, int32_t *out, cudaStream_t st, uint64_t *launches);
// With mag != null also the magnetisations [G][C][NT][32].
cudaError_t launch_energy(const uint32_t *spins, const uint32_t *bonds, int32_t *energy, int L,
                          uint32_t G, uint32_t NT, uint32_t C, cudaStream_t st,
                          uint64_t *launches, int32_t *mag = nullptr);
// Magnetisations of every lattice, out = DEVICE int32 [G][NT][C][32].
cudaError_t launch_magnetisation(const uint32_t *spins, int L, uint32_t G, uint32_t NT, uint32_t C,
                                 int32_t *out, cudaStream_t st, uint64_t *launches);
// Most threads a CTA of the external-field kernels has for lattice size L
// (384, so that a thread holds its 14 thresholds in registers; 512 for L = 32,
// whose lattices need 512 threads).
constexpr int field_max_threads(int L) { return L >= 32 ? 512 : 384; }
// External-field sweep kernels (ea_field.cu); called by launch_sweep_unit /
// launch_sweep_chunk when a.h_num != 0.
cudaError_t launch_sweep_unit_field(const SweepLaunch &a, int L, const Plan &plan, bool cluster_measure,
                                    cudaStream_t st);
cudaError_t launch_sweep_chunk_field(const SweepLaunch &a, int L, const Plan &plan, cudaStream_t st);
cudaError_t launch_measure(const uint32_t *spins, const int32_t *energy, int L, uint32_t G,
                           uint32_t NT, uint32_t C, int32_t *energies_out, uint32_t *ndiff_out,
                           uint64_t *qhist, int64_t *esum, cudaStream_t st, uint64_t *launches);

}  // namespace ea

// One ensemble's device state and counters (the opaque ea_ctx of the C ABI).
struct ea_ctx {
    uint32_t L, G, NT, C, N, swap_len;
    uint64_t seed;
    cudaStream_t stream;
    cudaMemPool_t pool;            // NULL: plain allocations; else stream-ordered from this pool
    int device;
    size_t smem_optin;
    uint32_t *d_spins, *d_bonds, *d_metro, *d_swapt, *d_masks;
    int32_t *d_energy;
    int *d_err;
    // external field h = h_num / h_den (h_num == 0: none, the pointers null)
    int32_t h_num, h_den, step;
    uint64_t *d_metro_f;           // [NT][2][7]
    int32_t *d_mag;                // [G][C][NT][32] magnetisations by slot
    uint32_t g_base;               // global index of group 0 (ea_config::group_base)
    uint64_t sweep, pass;
    uint64_t launches;
    std::vector<ea::Plan> plans;   // every kernel plan that can run this ensemble
    int plan_idx;
    ea::Plan plan;                 // plans[plan_idx]
    ea::RoundKeys rk;
};

namespace ea {
// Creates a context (ea_create with an optional memory pool: with a pool every
// allocation is stream-ordered on `stream` and nothing waits on the host).
// field: NULL, or the external field (ea_create_field).
int create_ctx(const ea_config *cfg, cudaStream_t stream, cudaMemPool_t pool, ea_ctx **out,
               const ea_field *field = nullptr);
// Releases a context's device memory (stream-ordered on `st` for pooled
// contexts) and the context itself.  The caller has ordered its last use.
void destroy_ctx(ea_ctx *c, cudaStream_t st);
// Device bytes create_ctx allocates for cfg, the import staging included.
size_t ctx_device_bytes(const ea_config *cfg);
// Temperature-packed contexts in the server: the stream their later work runs
// on, and the most device bytes ea_tp_create and ea_tp_sweep allocate for cfg
// (slot-group slices at eight groups a word included).
void tp_set_stream(ea_tp *t, cudaStream_t st);
size_t tp_device_bytes(const ea_tp_config *cfg);
}  // namespace ea
