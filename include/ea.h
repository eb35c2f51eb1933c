/*
 * ea.h -- C ABI of the GB300 (sm_103a) parallel-tempering Metropolis simulator
 * of the three-dimensional +-J Edwards-Anderson spin glass.
 *
 * The method is that of Fang et al., "Parallel Tempering Simulation of the
 * three-dimensional Edwards-Anderson Model with Compact Asynchronous Multispin
 * Coding on GPU": the Hamiltonian of Sec. 2.2 (Eq. 1, here with h = 0),
 * single-spin-flip Metropolis (Sec. 2.3) in a two-stage checkerboard sweep
 * (Sec. 3.1), replica exchange between adjacent temperatures (Sec. 2.4,
 * Sec. 4.1), integer threshold tables compared with the generator's integer
 * output (Sec. 4.3.1, 4.3.2), and measurements in their own pass (Sec. 4.1).
 *
 * Data conventions (every array is C order, little-endian uint32 words):
 *   L even >= 4, N = L^3 sites, site i = x + L*(y + L*z), periodic in x, y, z.
 *   G word-groups; bit b of a group's words is realization 32*g + b.
 *   NT temperature slots, slot 0 the coldest; C copies per slot (1 or 2).
 *   spins  [G][NT][C][N]  bit 1 <=> S = +1, indexed by temperature slot.
 *   bonds  [G][3][N]      bit 1 <=> J = -1 on bond (i, i + e_d), d = x, y, z.
 *   metro  [NT][3]        flip threshold for dE = 12 - 4u, u = 0, 1, 2;
 *                         each row non-decreasing in u.
 *   swapt  [NT-1][swap_len]  swap threshold for E_p - E_{p+1} = -4k at
 *                         column k-1; each row non-increasing in k.
 *   energies [G][NT][C][32] int32, E = -sum_bonds J S_i S_j (Eq. 1).
 * Random numbers: Philox4x32-10 keyed by seed = (lo32, hi32).
 *   Metropolis: one 32-bit output per (g, t, c, sweep s, site), shared by the
 *     32 realizations of the word: counter (k >> 2,
 *     (colour << 16) | (c << 8) | t, s, g), output word k & 3, k = i >> 1,
 *     colour = (x + y + z) & 1.
 *   Swap pass P, pair p, realization b: counter ((p << 3) | (b >> 2),
 *     (1 << 24) | (c << 8), P, g), output word b & 3.
 *   g is the global group index, ea_config::group_base + the group's index
 *     in the context's arrays.
 * A sweep updates colour 0 then colour 1.  Site i flips iff dE <= 0 or
 * r < metro[t][u], u = number of unsatisfied bonds of i.  After sweep s
 * (global index since creation) a swap pass runs iff swap_every > 0 and
 * (s + 1) % swap_every == 0: for each realization, pairs p = 0..NT-2 in
 * order, accept iff E_p - E_{p+1} >= 0 or r < swapt[p][k-1] with
 * k = (E_{p+1} - E_p) / 4 <= swap_len; an accepted pair exchanges the two
 * slots' configurations (that realization's bit only) and energies.
 *
 * Errors: every call returns EA_OK (0) or a negative EA_E* code; nothing is
 * thrown across the ABI.  Work is enqueued on the stream given at creation;
 * device faults surface as EA_ECUDA on the next call that synchronises
 * (ea_sync, ea_read_spins_host, ea_run, ea_get_*).  A context is not
 * thread-safe; use one per host thread.
 */
#ifndef EA_H
#define EA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EA_OK 0
#define EA_PENDING 1          /* ea_poll: request not finished yet */
#define EA_EINVAL (-1)        /* bad argument, shape, table or null pointer */
#define EA_ENOMEM (-2)        /* device or host allocation failed */
#define EA_ECUDA (-3)         /* CUDA runtime error (launch or device fault) */
#define EA_ETIMEOUT (-4)      /* wait deadline passed */
#define EA_EUNSUPPORTED (-5)  /* lattice size without a compiled kernel */
#define EA_ESTATE (-6)        /* call not valid in the object's current state */

typedef struct ea_ctx ea_ctx;

typedef struct {
    uint32_t L;               /* even, one of the sizes ea_supported_L() accepts */
    uint32_t n_groups;        /* G >= 1 (32 realizations each) */
    uint32_t n_temps;         /* 1 <= NT <= 64 */
    uint32_t n_copies;        /* C in {1, 2} */
    uint64_t seed;            /* Philox key */
    const uint32_t *bonds;    /* host [G][3][N], copied at creation */
    const uint32_t *spins0;   /* host [G][NT][C][N], copied at creation */
    const uint32_t *metro;    /* host [NT][3], copied */
    const uint32_t *swapt;    /* host [NT-1][swap_len], copied; may be NULL if swap_len == 0 */
    uint32_t swap_len;
    uint32_t group_base;      /* global index of word-group 0: group g of this context draws
                                 the random numbers of group group_base + g (the counters'
                                 fourth word), so contexts holding groups [b, b + G) of one
                                 ensemble reproduce exactly what those groups do in the whole
                                 ensemble (Sec. 3.3: realizations are independent jobs);
                                 group_base + G <= 2^32.  0 for a whole ensemble. */
} ea_config;

/* Options of one ea_sweep call.  All output pointers are DEVICE pointers and
 * may be NULL.  Counters continue from the context's global sweep index s and
 * swap-pass index P. */
typedef struct {
    uint32_t n_sweeps;
    uint32_t swap_every;      /* 0: no swap passes */
    int32_t *energy_log;      /* [n_sweeps][G][NT][C][32] energies by slot after each sweep
                                 (after its swap pass, if any) */
    uint32_t *swap_log;       /* [passes][G][C][NT-1] accepted-pair masks, bit b = realization b */
    uint64_t *qhist;          /* [NT][N+1] += 1 at bin n_diff for every (g, b) of each measured
                                 sweep; n_diff = #sites where copy 0 and copy 1 differ; needs C == 2 */
    int64_t *esum;            /* [NT] += sum over (g, c, b) of E at each measured sweep */
    uint64_t measure_from;    /* sweep s is measured iff s >= measure_from and */
    uint32_t measure_every;   /*   (s - measure_from) % measure_every == 0; 0 = never */
} ea_sweep_args;

/* Threshold tables in FP64 (Sec. 4.3.1, 4.3.2): metro[t][u] =
 * floor(exp(-beta_t (12 - 4u)) * 2^32) and swapt[p][k-1] =
 * floor(exp(-4k (beta_p - beta_{p+1})) * 2^32), clamped to 2^32 - 1.
 * beta: host [n_temps], >= 0 and non-increasing (slot 0 coldest).
 * swap columns run over k = 1..3N/2 (the largest possible |dE| / 4) with
 * trailing all-zero columns dropped; *swap_len_out receives that length.
 * swap_out (host [n_temps-1][swap_cap]) is filled when swap_cap >= the
 * length, else left untouched (call with swap_cap = 0 to query).
 * metro_out: host [n_temps][3], may be NULL.  Host-only, no GPU needed. */
int ea_build_tables(const double *beta, uint32_t n_temps, uint32_t n_sites, uint32_t *metro_out,
                    uint32_t *swap_out, uint32_t swap_cap, uint32_t *swap_len_out);

/* 1 if lattice size L has compiled kernels, else 0. */
int ea_supported_L(uint32_t L);

/* Allocates the device state of one ensemble on the current device and copies
 * the host arrays of cfg (the caller keeps ownership of them).  stream is a
 * cudaStream_t (NULL = legacy default stream); all later work of this context
 * is enqueued on it.  On success *out owns the context until ea_destroy. */
int ea_create(const ea_config *cfg, void *stream, ea_ctx **out);

/* Frees the context's device memory after its stream has drained.  NULL is a no-op. */
void ea_destroy(ea_ctx *ctx);

/* External field h = h_num / h_den: the Hamiltonian of Eq. 1 with the term
 * -h sum_i S_i (the field runs of Sec. 5).  With M = sum_i S_i, the method
 * works on Et = h_den (E - h M) = h_den E - h_num M, an integer:
 *   Metropolis: a flip of spin S with u unsatisfied bonds changes Et by
 *     h_den (12 - 4u) + 2 h_num S; it is accepted iff r < metro[t][S > 0][u]
 *     (uint64; 2^32 = always, the value where that change is <= 0).
 *   Swap pass: Et differences are multiples of step = gcd(4 h_den, 2|h_num|);
 *     pair p is accepted iff Et_p - Et_{p+1} >= 0 or r < swapt[p][k-1],
 *     k = (Et_{p+1} - Et_p) / step <= swap_len (cfg->swapt, cfg->swap_len
 *     are read in these units; cfg->metro is ignored and may be NULL).
 * Energies reported by the library stay E (bonds only, Eq. 1 at h = 0); the
 * field term is -h M with M from ea_magnetisations.  Requires h_den >= 1 and
 * (3 h_den + |h_num|) < 2^15 (Et differences fit int32 for N <= 32768).
 * h_num == 0 gives exactly the field-free method (metro[t][sp][u] must then
 * equal the field-free table for u < 3 and 2^32 above). */
typedef struct {
    int32_t h_num;
    int32_t h_den;
    const uint64_t *metro;    /* host [NT][2][7], each [t][sp] row non-decreasing in u, <= 2^32 */
} ea_field;

/* Field tables in FP64 (Sec. 4.3.1, 4.3.2 with the field term):
 * metro_out[t][sp][u] = floor(exp(-beta_t (12 - 4u + 2 h S)) 2^32) (clamped
 * below 2^32) where that energy change is > 0, else 2^32; S = +1 for sp = 1.
 * swap columns k = 1..(6N h_den + 2N |h_num|) / step hold
 * floor(exp(-(beta_p - beta_{p+1}) k step / h_den) 2^32) with trailing zero
 * columns dropped; *swap_len_out, swap_cap and swap_out as ea_build_tables.
 * Host-only. */
int ea_build_tables_field(const double *beta, uint32_t n_temps, uint32_t n_sites, int32_t h_num,
                          int32_t h_den, uint64_t *metro_out, uint32_t *swap_out, uint32_t swap_cap,
                          uint32_t *swap_len_out);

/* ea_create in the field `field` (NULL: none, as ea_create).  Contexts with a
 * field run the generic unit and chunked kernel forms, and at L = 8 the
 * wavefront form when the field's always-accept boundaries are u >= 3 for one
 * spin value and u >= 4 for the other (0 < |h| < 2 with the builder's tables).
 * A batch takes members all in a field or all field-free (EA_EINVAL when
 * mixed); its field members run in a field kernel of 384-thread CTAs. */
int ea_create_field(const ea_config *cfg, const ea_field *field, void *stream, ea_ctx **out);

/* Magnetisations M = sum_i S_i of every lattice by slot, recomputed from the
 * spins: DEVICE int32 [G][NT][C][32].  Any context.  Asynchronous. */
int ea_magnetisations(ea_ctx *ctx, int32_t *out);

/* Runs args->n_sweeps sweeps of the method: each a two-stage checkerboard
 * sweep (Sec. 3.1: colour 0, then colour 1) of single-spin-flip Metropolis
 * updates (Sec. 2.3; flip iff r < metro[t][u] or dE <= 0, Sec. 4.3.1-4.3.2),
 * followed by the replica-exchange pass of Sec. 2.4 when (s + 1) % swap_every
 * == 0, and the measurements the arguments ask for (Sec. 4.1).  Outputs and
 * their layouts are those of ea_sweep_args (DEVICE pointers).  EA_EINVAL for
 * a NULL context or arguments, or a qhist with one copy.
 * Asynchronous on the context's stream; device faults surface at the next
 * synchronising call. */
int ea_sweep(ea_ctx *ctx, const ea_sweep_args *args);

/* One replica-exchange pass now (Sec. 2.4; pass index P, then P += 1) on
 * energies recomputed from the spins: for each realization, pairs p = 0..NT-2
 * in order, accepted iff E_p - E_{p+1} >= 0 or r < swapt[p][k-1] (Sec. 4.3.2),
 * an accepted pair exchanging the slots' configurations and energies.
 * masks: DEVICE [G][C][NT-1] (bit b = realization b accepted pair p) or NULL.
 * EA_EINVAL for a NULL context.  Asynchronous. */
int ea_pt_swap(ea_ctx *ctx, uint32_t *masks);

/* Measurement pass (Sec. 4.1): recomputes the energies from the spins.
 * energies: DEVICE [G][NT][C][32] int32 or NULL; ndiff: DEVICE [G][NT][32]
 * uint32 or NULL (needs C == 2); qhist: DEVICE [NT][N+1] uint64, += one
 * count per (g, b), or NULL (needs C == 2).  Asynchronous. */
int ea_measure(ea_ctx *ctx, int32_t *energies, uint32_t *ndiff, uint64_t *qhist);

/* Per-plane counts for Fourier-mode observables (Sec. 5: the spin-glass
 * correlation length from the overlap, the ferromagnet's from the
 * magnetisation).  Site i = x + L(y + Lz); plane (axis a, index p) holds the
 * L^2 sites whose a-th coordinate (x, y, z for a = 0, 1, 2) is p.
 * mode 0: sites of each plane where the two copies of a slot differ,
 *         out = DEVICE int32 [G][NT][3][L][32] (needs n_copies == 2);
 * mode 1: up spins of each plane per copy, out = DEVICE int32 [G][NT][C][3][L][32].
 * Asynchronous on the context's stream; EA_EINVAL for another mode or mode 0
 * with one copy. */
int ea_measure_planes(ea_ctx *ctx, int mode, int32_t *out);

/* Spins by temperature slot (the configuration of Eq. 1 each slot holds
 * after the exchanges of Sec. 2.4) into DEVICE dst [G][NT][C][N], bit 1 <=>
 * S = +1, site order of the data conventions above.  The caller owns dst.
 * EA_EINVAL for a NULL context or dst.  Asynchronous. */
int ea_read_spins(ea_ctx *ctx, uint32_t *dst);

/* As ea_read_spins into HOST dst [G][NT][C][N]; synchronises the stream
 * (EA_ECUDA if a device fault is pending). */
int ea_read_spins_host(ea_ctx *ctx, uint32_t *dst);

/* Replaces the state (checkpoint restore): spins from DEVICE src
 * [G][NT][C][N] by slot (layout of ea_read_spins; the caller keeps src), and
 * the global sweep and swap-pass indices that the counters of Sec. 4.3.2's
 * generator continue from; energies are recomputed from the spins (Eq. 1).
 * EA_EINVAL for a NULL context or src.  Asynchronous. */
int ea_write_spins(ea_ctx *ctx, const uint32_t *src, uint64_t sweep_index, uint64_t pass_index);

/* Global sweep index s of the next sweep and pass index P of the next swap pass. */
int ea_get_counters(const ea_ctx *ctx, uint64_t *sweep_index, uint64_t *pass_index);

/* Waits for the context's stream; returns EA_ECUDA on a device fault and
 * EA_ETIMEOUT (clearing it) if a kernel's bounded wait between its warps ran
 * out since the last check (it never should; the state is then not advanced
 * consistently and must be rewritten with ea_write_spins). */
int ea_sync(ea_ctx *ctx);

/* Number of kernel launches this context has enqueued so far. */
uint64_t ea_launch_count(const ea_ctx *ctx);

/* Kernel plans.  An ensemble can run under several plans (kernel form, CTA
 * shape, shared-memory staging); all give bit-identical results and differ
 * only in speed.  ea_create selects a default; ea_autotune times them. */
typedef struct {
    int32_t form;              /* 0: unit (all slots of a group and copy in one CTA, generic);
                                  1: unit, specialised for L % 8 == 0;
                                  2: chunked (slots split over CTAs, swap pass as own kernels) */
    int32_t threads;           /* threads per CTA */
    int32_t group_threads;     /* threads per lattice (form 1: per lattice row-parity class) */
    int32_t lattices_per_cta;
    uint64_t smem_bytes;       /* dynamic shared memory per CTA */
    int32_t units_per_cta;     /* unit forms: (group, copy) units a CTA runs in lockstep (1
                                  outside batches); chunked: 0 */
} ea_plan_desc;

int ea_plan_count(const ea_ctx *ctx);
int ea_plan_current(const ea_ctx *ctx);
int ea_plan_info(const ea_ctx *ctx, int index, ea_plan_desc *out);
int ea_plan_select(ea_ctx *ctx, int index);

/* Autotuner: runs every plan twice for probe_sweeps sweeps (swap pass every
 * swap_every) from the current state, restoring the state after each run,
 * and selects the fastest.  Spins, energies and counters are unchanged.
 * ms_out: host [ea_plan_count] receives the second run's milliseconds (may
 * be NULL).  Synchronises the stream. */
int ea_autotune(ea_ctx *ctx, uint32_t probe_sweeps, uint32_t swap_every, float *ms_out);

/* Batched form: one persistent launch advances several ensembles together.
 *
 * A batch holds contexts (any supported L, ladder and size, on one device).
 * ea_batch_sweep advances every member by n sweeps with the given swap
 * schedule; each member's trajectory, energies and counters are exactly those
 * of ea_sweep on it alone (same random-number counters), without logs or
 * measurements.  The work of all members is cut into tasks -- whole
 * (group, copy) units resident in one CTA for a segment of sweeps, or slot
 * chunks of units too large for one CTA for one swap interval, whose last
 * chunk runs the unit's swap pass -- and run by one persistent launch from a
 * device-side queue, longest unit first.  The paper simulates one ensemble at
 * a time (Sec. 3); batching several is this library's own addition, and the
 * arithmetic of each member is that of Sec. 2.3 (sweeps) and Sec. 2.4 (swaps)
 * exactly as in ea_sweep.  A call whose shape (members, tasks, shared
 * memory, width) repeats the previous call's is captured in a CUDA graph
 * (upload, queue reset, launch) and replayed while the shape stays the same;
 * other calls launch directly.  Asynchronous on the batch's stream (NULL = legacy default);
 * members must not be used on other streams until ea_batch_sync returns.
 * A device-side wait that runs out (it never should) makes ea_batch_sync
 * return EA_ETIMEOUT instead of hanging. */
typedef struct ea_batch ea_batch;
int ea_batch_create(void *stream, ea_batch **out);
/* ctx must outlive its membership; adding a member twice is EA_EINVAL. */
int ea_batch_add(ea_batch *batch, ea_ctx *ctx);
int ea_batch_clear(ea_batch *batch);
/* Plans a member can run under inside the batch kernel (its own list, made
 * for CTAs of up to 512 threads: the L % 8 == 0 unit kernel, the generic unit
 * body with several lockstep units per CTA, balanced slot chunks).  All give
 * bit-identical results.  ea_batch_plan_current: the plan the next call uses
 * (the explicit choice, else a default that keeps the most threads busy). */
int ea_batch_plan_count(const ea_batch *batch, uint32_t member);
int ea_batch_plan_info(const ea_batch *batch, uint32_t member, int index, ea_plan_desc *out);
int ea_batch_plan_current(const ea_batch *batch, uint32_t member);
/* Selects a member's plan by index into its batch list; -1 = automatic. */
int ea_batch_set_plan(ea_batch *batch, uint32_t member, int plan_index);
/* Width of the batch kernel: 384 or 512 threads a CTA, 0 = automatic (384
 * unless a chosen plan needs more).  Plans wider than the width fail the
 * next ea_batch_sweep with EA_EUNSUPPORTED. */
int ea_batch_set_width(ea_batch *batch, int threads);
/* How long a CTA of the batch kernel waits for its next task before it
 * raises the batch's error flag (in naps of ~256 ns; 0 = the default, tens
 * of seconds).  A call whose wait runs out ends with every CTA returned and
 * ea_batch_sync reporting EA_ETIMEOUT; the members' state is then partly
 * advanced and must be rewritten (ea_write_spins) or discarded.  Correct
 * calls never wait that long. */
int ea_batch_set_wait_limit(ea_batch *batch, uint32_t naps);
/* Test hook for that path: the next ea_batch_sweep queues one task that is
 * never published, so one CTA's wait runs out (no fault, no trap). */
int ea_batch_inject_stall(ea_batch *batch);
/* Work of one unit task in site-word updates (sweeps x N x NT x units); 0 = default. */
int ea_batch_set_segment(ea_batch *batch, uint32_t site_words);
int ea_batch_sweep(ea_batch *batch, uint32_t n_sweeps, uint32_t swap_every);
/* Per-member sweeps: member i advances n_sweeps[i] sweeps (0: left out of
 * this call) with its own swap_every[i] (host arrays of the member count). */
int ea_batch_sweep_each(ea_batch *batch, const uint32_t *n_sweeps, const uint32_t *swap_every);
int ea_batch_sync(ea_batch *batch);
/* Batch autotuner: for each kernel width, a coordinate descent over every
 * member's plans, each probe a warm call and a timed call of probe_sweeps
 * sweeps of the whole batch from the current state (restored after each
 * call); keeps the fastest width and plans.  Spins, energies and counters are
 * unchanged.  best_ms (may be NULL) receives the best probe's milliseconds.
 * Allocates a copy of every member's state while it runs; synchronises. */
int ea_batch_autotune(ea_batch *batch, uint32_t probe_sweeps, uint32_t swap_every, float *best_ms);
uint64_t ea_batch_launch_count(const ea_batch *batch);
void ea_batch_destroy(ea_batch *batch);

/* Serving loop: a server accepts simulation requests from any thread, admits
 * them in arrival order while their device memory fits its budget, keeps
 * their state resident, and advances resident requests together in rounds
 * of one batched launch (ea_batch_sweep_each), each by up to the number of
 * sweeps that makes the round last about round_ms; requests that arrive
 * meanwhile join at the next round (continuous batching).  A round takes the
 * requests with the least work left, in that order, until their (group,
 * copy) units give about two tasks per SM (shortest remaining work first
 * while the GPU stays full); a request left out of 64 consecutive rounds
 * goes first.  Each
 * result is exactly what ea_create + ea_sweep would give alone.  The paper
 * runs one simulation at a time (Sec. 3); serving is this library's own
 * addition.  One worker thread per server owns its GPU work; the server uses
 * the device that is current at ea_server_create. */
typedef struct ea_server ea_server;
typedef struct {
    uint64_t mem_budget;       /* device bytes for resident requests; 0 = 81% of free memory
                                  (never more than 90% of free memory at creation) */
    uint32_t max_live;         /* most resident requests; 0 = 256 */
    uint32_t round_ms;         /* target duration of a round; 0 = 20 */
} ea_server_opts;
int ea_server_create(const ea_server_opts *opts, ea_server **out);   /* opts may be NULL */

typedef struct {
    uint32_t n_sweeps, swap_every;
    uint32_t *spins_out;       /* HOST [G][NT][C][N] final spins (slot order), or NULL */
    int32_t *energies_out;     /* HOST [G][NT][C][32] final energies E (Eq. 1, bonds), or NULL */
    int32_t *magnetisations_out;   /* HOST [G][NT][C][32] final M, or NULL; requests in a
                                      field only (ea_submit_field with h_num != 0) */
} ea_request;
/* Copies cfg's host inputs and queues the request; *ticket identifies it.
 * The output buffers must stay valid until ea_poll reports it finished.
 * Shape errors return at once (EA_EINVAL / EA_EUNSUPPORTED); table errors
 * and a request larger than the whole budget (EA_ENOMEM) finish the ticket. */
int ea_submit(ea_server *server, const ea_config *cfg, const ea_request *req, uint64_t *ticket);
/* ea_submit in the external field `field` (as ea_create_field; cfg->metro may
 * then be NULL).  Requests in a field advance in the server's field batches
 * (one persistent launch per round for them, beside the field-free one); the
 * field's tables are copied.  Each result is exactly what ea_create_field +
 * ea_sweep would give alone. */
int ea_submit_field(ea_server *server, const ea_config *cfg, const ea_field *field, const ea_request *req,
                    uint64_t *ticket);
/* Waits up to timeout_us for the ticket: EA_PENDING if unfinished; else the
 * request's status (EA_OK: outputs written), after which the ticket is
 * retired and polling it again is EA_EINVAL. */
int ea_poll(ea_server *server, uint64_t ticket, uint32_t timeout_us);
typedef struct {
    uint64_t submitted, completed, failed, queued, live, rounds;
    double p50_ms, p99_ms, mean_ms, max_ms;   /* completion latency: submit -> outputs written */
    double flip_attempts;      /* of completed requests: N x NT x C x 32G x sweeps */
    double busy_s;             /* time with at least one request resident */
    double span_s;             /* first submission -> last completion */
    uint64_t mem_budget, peak_bytes;   /* budget and most device bytes resident at once */
} ea_server_stats;
int ea_server_stats_get(ea_server *server, ea_server_stats *out);
/* Stops the worker; requests not yet finished are dropped. */
void ea_server_destroy(ea_server *server);

/* Host-buffer entry point: creates a context from cfg, runs the sweeps of
 * args (its DEVICE output pointers must be NULL), copies the results to the
 * HOST buffers below (each may be NULL), destroys the context and
 * synchronises.  Host outputs: energies [G][NT][C][32] (final), spins
 * [G][NT][C][N] (final), qhist [NT][N+1] (overwritten with this run's counts),
 * esum [NT] (overwritten).  stream as in ea_create. */
int ea_run(const ea_config *cfg, const ea_sweep_args *args, void *stream, int32_t *energies_host,
           uint32_t *spins_host, uint64_t *qhist_host, int64_t *esum_host);

/* One replica-exchange pass that allocates no device memory.  The paper has
 * no counterpart: this exists for callers that cannot call cudaMalloc while
 * they run (an application that pre-reserves all device memory for its own
 * pool, a host thread that must not stall other streams on an allocation).
 * It performs the field-free pass of ea_pt_swap (h = 0: the decision is
 * E_p - E_{p+1} >= -4k against swapt; contexts made with a field decide on
 * Et instead and must not use it) on caller-owned DEVICE buffers:
 *   spins    [G][NT][C][N] by slot (the layout of ea_read_spins), exchanged in place;
 *   energies [G][NT][C][32] int32 of those spins (as ea_measure returns them),
 *            permuted in place to follow the exchanged configurations;
 *   swapt    DEVICE [NT-1][swap_len], the table of ea_build_tables;
 *   masks    DEVICE [G][C][NT-1] or NULL.
 * seed and pass_index give the random numbers (pass P of the context API);
 * group g of the buffers draws those of group g (group_base 0).
 * Its scratch (the accepted-pair masks between its two kernels) is a static
 * device array of the library sized for G * C <= 4096; larger ensembles, and
 * L with L^3 >= 2^32, get EA_EINVAL.  The first call on each device looks up
 * that array's device address and keeps it for the process (make that call
 * before any stream capture; after a cudaDeviceReset the address is stale and
 * this call must not be used).  Every call shares the array: calls whose
 * kernels overlap on the GPU (other streams, other host threads) race; calls
 * on one stream are ordered.  Asynchronous on stream. */
int ea_pt_swap_static(uint32_t *spins, int32_t *energies, const uint32_t *swapt, uint32_t swap_len,
                      uint32_t L, uint32_t n_groups, uint32_t n_temps, uint32_t n_copies,
                      uint64_t seed, uint64_t pass_index, uint32_t *masks, void *stream);

/* ---- Temperature-packed form ------------------------------------------------
 * The word layout of the paper's compact asynchronous multispin coding
 * (Sec. 3.2 "Map Temperatures Replicas to Bits", Sec. 4.3.3): one 32-bit word
 * per (realization, copy, site) whose bit t is the spin of temperature slot t,
 * so the temperature replicas of one realization are updated together and a
 * replica exchange (Sec. 2.4) permutes bits inside each word.  NT <= 32
 * takes one word per site; 33 <= NT <= 64 takes two (slot 32 w + b in bit b
 * of word w, the paper's several integer cubes).
 *
 * Random numbers: each realization has its own.  Realization r uses the
 * counters of word-group r of the realization-packed form above (bit 0 of
 * that group): Metropolis uniform of (r, slot t, copy c, sweep s, site i) =
 * output k & 3 of Philox(k >> 2, (colour << 16) | (c << 8) | t, s, r), swap
 * uniform of pair p in pass P = output 0 of Philox(p << 3, (1 << 24) | (c << 8),
 * P, r).  Everything else (tables, sweep order, swap rule, energies) is the
 * method above, so realization r follows exactly the trajectory of realization
 * 32r of a realization-packed ensemble with the same bonds, spins and tables.
 * This form spends one uniform per flip attempt instead of one per 32; it
 * suits ensembles with few realizations and many temperatures.
 */
typedef struct ea_tp ea_tp;

typedef struct {
    uint32_t L;               /* as ea_config (ea_supported_L) */
    uint32_t n_real;          /* R >= 1 realizations */
    uint32_t n_temps;         /* 1 <= NT <= 64: W = ceil(NT / 32) words per site */
    uint32_t n_copies;        /* C in {1, 2} */
    uint64_t seed;            /* Philox key */
    const uint8_t *bonds;     /* host [R][3][N]: nonzero <=> J = -1 on bond (i, i + e_d); copied */
    const uint32_t *spins0;   /* host [R][C][W][N]: bit b of word w <=> S = +1 in slot 32 w + b (the
                                 paper's several integer cubes, Sec. 3.2); bits of slots >= NT ignored;
                                 copied */
    const uint32_t *metro;    /* host [NT][3] as ea_config; copied */
    const uint32_t *swapt;    /* host [NT-1][swap_len] as ea_config; copied */
    uint32_t swap_len;
    uint32_t real_base;       /* global index of realization 0: realization r draws the random
                                 numbers of realization real_base + r (as ea_config::group_base);
                                 real_base + R <= 2^32.  0 for a whole ensemble. */
} ea_tp_config;

/* Validates cfg (EA_EINVAL on a bad shape or table, EA_EUNSUPPORTED on L),
 * allocates the device state, imports the inputs and computes the initial
 * energies on `stream` (a cudaStream_t, NULL = legacy default stream), and
 * synchronises that stream once.  *out is owned by the caller until
 * ea_tp_destroy. */
int ea_tp_create(const ea_tp_config *cfg, void *stream, ea_tp **out);
/* n_sweeps sweeps, each followed by a swap pass iff swap_every > 0 and
 * (s + 1) % swap_every == 0 (s global), in one kernel launch.  DEVICE outputs,
 * each may be NULL: energy_log [n_sweeps][R][NT][C] int32 (energies by slot
 * after each sweep and its pass), swap_log [passes][R][C][W] uint32 (bit b of
 * word w = pair 32 w + b accepted).  One launch for the whole call when W = 1
 * and the unit is not split into slot groups; otherwise two launches per swap
 * interval (the groups' sweeps, then the merge with the pass).  Asynchronous
 * on the context's stream. */
int ea_tp_sweep(ea_tp *tp, uint32_t n_sweeps, uint32_t swap_every, int32_t *energy_log,
                uint32_t *swap_log);
/* Copies the state to DEVICE buffers, each may be NULL: spins [R][C][W][N]
 * (bit b of word w = slot 32 w + b, bits of slots >= NT zero), energies
 * [R][NT][C] int32.  Asynchronous. */
int ea_tp_read(ea_tp *tp, uint32_t *spins, int32_t *energies);
/* Global sweep and pass indices, the number of kernels launched so far and
 * the number of slot groups per (realization, copy) unit (each pointer may be
 * NULL). */
int ea_tp_info(const ea_tp *tp, uint64_t *sweep_index, uint64_t *pass_index, uint64_t *launches,
               uint32_t *split);
/* Splits each word of each (realization, copy) unit into k slot groups (k a
 * power of two, 1 <= k <= min(32, NT); groups of ceil(min(NT, 32) / k) slots,
 * the ones empty in the first word dropped), one CTA each: slots do not
 * interact between swap passes, so every group sweeps its own slots up to the
 * next pass and a merge launch then combines the groups and runs the pass.
 * Results do not depend on k.  ea_tp_create picks the largest k <= 8 with
 * R * C * W * k CTAs within one per SM (1 when R * C * W fills the GPU).  May
 * allocate device memory (one word per site and group); synchronises the
 * stream when it frees some.  EA_EINVAL for another k.  ea_tp_info reports the
 * groups in use per unit (W times the groups per word). */
int ea_tp_set_split(ea_tp *tp, uint32_t k);
/* Synchronises the context's stream and frees its device memory. */
void ea_tp_destroy(ea_tp *tp);

/* A temperature-packed request to the server (see ea_submit_tp). */
typedef struct {
    uint32_t n_sweeps, swap_every;   /* as ea_tp_sweep */
    uint32_t *spins_out;       /* HOST [R][C][W][N] final words (ea_tp_read's layout), or NULL */
    int32_t *energies_out;     /* HOST [R][NT][C] final energies by slot, or NULL */
} ea_tp_request;
/* Queues a temperature-packed request (Sec. 3.2's word layout, the ea_tp_*
 * context above) on the server: cfg's host inputs are copied, the request is
 * admitted by device memory like any other, and each round advances it on the
 * server's compute stream behind the round's batched launches (one launch, or
 * the slot groups and their merge, per round).  Its result is exactly what
 * ea_tp_create + ea_tp_sweep(n_sweeps, swap_every) + ea_tp_read give alone.
 * Shape errors return at once (EA_EINVAL / EA_EUNSUPPORTED); table errors and
 * a request larger than the whole budget finish the ticket.  Creating and
 * destroying such a context allocates and frees with cudaMalloc / cudaFree,
 * which synchronise the device: rounds that admit or finish one do not overlap
 * the next round. */
int ea_submit_tp(ea_server *server, const ea_tp_config *cfg, const ea_tp_request *req, uint64_t *ticket);

/* Static description of an error code. */
const char *ea_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* EA_H */
