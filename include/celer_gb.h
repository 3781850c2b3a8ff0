/*
 * celer_gb -- step-based electromagnetic Monte Carlo transport on one GB300.
 *
 * C ABI of the library. The method is the step-based ("per-action") stepping
 * loop of Sec. 2 of Lund et al., "Accelerating detector simulations with
 * Celeritas: profiling and performance optimizations" (arXiv:2503.17608):
 * active tracks live in a structure-of-arrays slot store, each step iteration
 * first fills vacant slots from a buffer of track initializers, then applies
 * one action at a time (step limit, propagation, discrete interaction) to
 * all tracks as separate kernel launches; secondaries go back into the
 * initializer buffer. Sec. 3.1 adds reordering of track-slot indices by
 * action so that each action kernel sees tracks doing the same thing; here
 * that reordering is a stable radix partition, and each action kernel runs
 * over one contiguous range of the partition.
 *
 * Conventions for every entry point:
 *   - the return value is a celer_status; no call aborts, traps or exits;
 *   - device work is ordered on the CUDA stream given in celer_problem;
 *     calls that return data to the host synchronise that stream only;
 *   - the context owns all device memory and all pinned host staging
 *     memory it allocates in celer_create; the caller owns every host array
 *     it passes and may reuse it as soon as the call returns;
 *   - a context is not thread safe: one host thread at a time;
 *   - after CELER_ERR_CUDA the context must be destroyed; after any other
 *     error it stays usable.
 *
 * Units: MeV, cm, tesla, g/cm3.
 */
#ifndef CELER_GB_H
#define CELER_GB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CELER_OK = 0,
  CELER_ERR_INVALID = 1,   /* bad argument; nothing was changed */
  CELER_ERR_CAPACITY = 2,  /* a fixed-size buffer would overflow; state is intact */
  CELER_ERR_CUDA = 3,      /* a CUDA call failed; destroy the context */
  CELER_ERR_TIMEOUT = 4,   /* the iteration limit was reached; state is intact */
  CELER_ERR_STATE = 5      /* call not allowed in the current state */
} celer_status;

/* particle types (the "particle type" field of the track state, Sec. 2) */
enum { CELER_GAMMA = 0, CELER_ELECTRON = 1, CELER_POSITRON = 2 };

/* process bitmask */
enum {
  CELER_PROC_COMPTON = 1,
  CELER_PROC_PHOTOELECTRIC = 2,
  CELER_PROC_PAIR = 4,
  CELER_PROC_MOLLER = 8,
  CELER_PROC_BREMS = 16,
  CELER_PROC_ELOSS = 32
};

/* tally layouts: uniform z bins over the world, or one bin per layer */
enum { CELER_TALLY_ZBINS = 0, CELER_TALLY_LAYERS = 1 };

/* Track-reordering policies (Sec. 3.1, "Reindexing track slots", and
 * Sec. 3.2, "Partitioning track data"):
 *   NONE        every action kernel runs over all slots and masks the tracks
 *               that do not take part (Sec. 2, "masking");
 *   ACTION      slot indices are partitioned by along-step action (neutral
 *               straight line vs charged), the key the paper found best;
 *   ACTION_TYPE slot indices are partitioned by (particle type, next action),
 *               so every along-step and interaction kernel runs over one
 *               contiguous range;
 *   LOCAL       no grid-wide partition: in the step phase each GPU block
 *               groups its own live tracks by (particle type, next action) in
 *               on-chip memory and gives each warp one group (no counterpart
 *               in the paper; it keeps the divergence cut of ACTION_TYPE
 *               without the partition's extra grid-wide pass). The per-action
 *               launch mode runs it like NONE.
 *   DATA        no reindexing (Sec. 3.2): the initializers that fill vacant
 *               slots are partitioned by charge, the neutral ones placed at the
 *               low end and the charged ones at the high end of each GPU
 *               block's share of the slot array, and the tracks are stepped in
 *               slot order with masking. The per-action launch mode runs it
 *               like NONE.
 * LOCAL and DATA fill the slots block by block (each block's lowest vacant
 * slots, DATA: lowest and highest, take an even share of the initializers);
 * the other policies fill the r-th vacant slot in slot order with the r-th
 * queued initializer. Either way the fill is deterministic, and results do not
 * depend on it (random streams follow the track, not the slot). */
enum { CELER_SORT_NONE = 0, CELER_SORT_ACTION = 1, CELER_SORT_ACTION_TYPE = 2, CELER_SORT_LOCAL = 3,
       CELER_SORT_DATA = 4 };

typedef struct {
  double Z;       /* atomic number (effective Z for a compound) */
  double A;       /* g/mol; unused when ne > 0 */
  double rho;     /* g/cm3 */
  double ne;      /* electrons / cm3; 0: derived as N_A rho Z / A */
  double X0;      /* radiation length, cm */
  double I;       /* mean excitation energy, MeV */
} celer_material;

typedef struct {
  int n_materials;
  const celer_material* materials;   /* host, n_materials entries; copied */
  int n_layers;                      /* slabs in one period along z */
  const int* layer_material;         /* host, n_layers; material index per slab */
  const double* layer_thickness;     /* host, n_layers; cm, > 0 */
  int n_periods;                     /* the period is repeated this many times from z = 0 */
  double half_x, half_y;             /* transverse half-widths of the world, cm */
  double Bz;                         /* uniform field along z, tesla (0: none) */
  double cut_track;                  /* tracking cut, all particles, MeV (>= 1 keV) */
  double cut_moller;                 /* delta-ray production cut, MeV */
  double cut_brems;                  /* bremsstrahlung photon production cut, MeV */
  int processes;                     /* CELER_PROC_* bitmask */
  int tally_mode;                    /* CELER_TALLY_* */
  int n_zbins;                       /* bins for CELER_TALLY_ZBINS */
  uint64_t n_slots;                  /* track slots (the state size of Sec. 2) */
  uint64_t init_capacity;            /* initializer buffer entries (rounded up to a power of two) */
  uint32_t max_events;               /* tally rows; event e uses row e % max_events */
  uint64_t history_capacity;         /* per-primary records (0: off) */
  int sort_policy;                   /* CELER_SORT_* */
  int block_size;                    /* threads per block of the action kernels: 128, 256 or 512 */
  int split_actions;                 /* 1: one launch per along-step / interaction action (host and
                                        graph loops); 0: one launch per phase covering all actions */
  uint32_t seed;                     /* first word of every Philox key */
  uint64_t max_iterations;           /* celer_run_events limit (0: 10^6) */
  void* cuda_stream;                 /* cudaStream_t for all work (NULL: legacy default stream) */
  int field_substep_cap;             /* charged tracks in the field (Sec. 3.3): 0 the exact helix;
                                        > 0 classical Runge-Kutta substeps of at most 0.1 rad of
                                        turn, at most this many per step: a longer step is cut
                                        there and ends without crossing or interaction (action
                                        "field"), to go on at the next iteration; < 0 invalid */
} celer_problem;

typedef struct {
  double E;        /* kinetic energy, MeV, in (0, 10^4] */
  double pos[3];   /* cm, inside the world */
  double dir[3];   /* unit vector, |dir| = 1 within 1e-12 */
  int32_t ptype;   /* CELER_GAMMA or CELER_ELECTRON */
  int32_t pad;
} celer_primary;

typedef struct {
  uint64_t iteration;        /* step iterations completed so far */
  uint64_t alive;            /* tracks in slots after this iteration */
  uint64_t queued;           /* initializers waiting after this iteration */
  uint64_t steps;            /* track-steps taken in this iteration */
  uint64_t steps_total;      /* track-steps since creation */
  uint32_t deferred;         /* interactions postponed for lack of buffer space */
  uint32_t error;            /* device error bits (0: none) */
  uint32_t action_count[16]; /* tracks per next action in this iteration */
} celer_step_stats;

typedef struct {
  uint64_t steps;        /* track-steps of the primary and all its descendants */
  uint64_t secondaries;  /* secondary tracks created above the tracking cut */
  double escaped;        /* energy that left the world, MeV */
  double edep;           /* energy deposited, MeV (sum over bins) */
} celer_history;

typedef struct {
  uint64_t iteration, alive, queued, steps;
  uint32_t action_count[16];
} celer_trace_row;

typedef struct celer_ctx celer_ctx;

/* Human-readable name of a status code (static string). */
const char* celer_status_string(celer_status s);

/* Message of the last error on this context (static per context; "" if none). */
const char* celer_last_error(const celer_ctx* ctx);

/* Build a context (Sec. 2: the state of the active tracks is a struct of
 * arrays with one entry per track slot, and new tracks wait in a separate
 * buffer of track initializers): validate the problem, allocate the slot
 * store (n_slots slots, one device array per field), the initializer buffer
 * (init_capacity entries), tallies and history on the current CUDA device,
 * and build the cross-section, stopping-power and range tables on the
 * device. problem: host, read during the call only. *out receives the
 * context, or NULL on error; the caller releases it with celer_destroy.
 * CELER_ERR_INVALID for an inconsistent problem (nothing allocated),
 * CELER_ERR_CUDA if an allocation or launch fails (everything allocated so
 * far is released). */
celer_status celer_create(const celer_problem* problem, celer_ctx** out);

/* Release every resource of the context (Sec. 2: the track-slot store and
 * the initializer buffer, with the tables, tallies and pinned staging
 * memory): synchronises the context's stream, then frees. NULL is allowed;
 * the pointer is invalid afterwards. */
void celer_destroy(celer_ctx* ctx);

/* Queue n primaries of one event as track initializers (Sec. 2: new tracks
 * enter through the initializer buffer). host_ptr: n celer_primary records in
 * host memory (pageable or pinned). The i-th primary added to an event gets
 * track id = number of primaries of that event added before it, which keys
 * its random stream together with (seed, event). Validation happens on the
 * host before any device work: CELER_ERR_INVALID for a bad record,
 * CELER_ERR_CAPACITY if the initializer buffer or history cannot hold them.
 * Reads the buffer fill level from the device (one stream synchronisation)
 * only if step work has run since it was last read; consecutive calls between
 * two runs (a serving loop admitting several events) synchronise at most
 * once. */
celer_status celer_add_primaries(celer_ctx* ctx, uint32_t event, const celer_primary* host_ptr, uint64_t n);

/* Same as celer_add_primaries for n records already in device memory
 * (device_ptr: n celer_primary records on the context's device, e.g. a
 * CUDA tensor). Validation and the initializer-buffer capacity check run on
 * the device, stream ordered, without a host round trip: if any record is
 * invalid or the buffer cannot hold all n, none is queued and the next call
 * that synchronises (celer_run_events, celer_step with stats,
 * celer_get_stats) reports CELER_ERR_INVALID. Track ids are assigned as in
 * celer_add_primaries, whether or not the batch is accepted. The caller
 * keeps device_ptr valid until the stream has passed this call. */
celer_status celer_add_primaries_device(celer_ctx* ctx, uint32_t event, const celer_primary* device_ptr, uint64_t n);

/* One step iteration (Sec. 2): fill vacant slots from initializers, step
 * limit, reorder (Sec. 3.1, per sort_policy), propagation, interactions,
 * secondaries to the initializer buffer. If stats is non-NULL the stream is
 * synchronised and the iteration's counters are returned. */
celer_status celer_step(celer_ctx* ctx, celer_step_stats* stats);

/* Loop modes of celer_run_events. */
enum {
  CELER_LOOP_HOST = 0,       /* host loop of per-iteration launches, polling the counters every few iterations */
  CELER_LOOP_GRAPH = 1,      /* the iteration captured once into a CUDA graph whose conditional while-node
                                repeats it on the device with no host round trip */
  CELER_LOOP_PERSISTENT = 2, /* one cooperative launch that runs every iteration: one block per SM slot,
                                tables staged into shared memory once, phases separated by grid barriers
                                whose waits are bounded (about 1 s, then CELER_ERR_TIMEOUT) */
  CELER_LOOP_ASYNC = 3       /* block-pass policies (CELER_SORT_LOCAL, CELER_SORT_DATA) only: one cooperative
                                launch in which every block runs its own step iterations ("passes") over its
                                own slots with no grid barrier, sharing the initializer buffer as a
                                concurrent queue (a block takes ceil(queued / blocks) entries per pass, at
                                most its vacant slots; an entry's state word orders its writer and its
                                reader). Histories are those of the synchronous modes (every track's random
                                stream is keyed by its own id); tallies differ only in summation order.
                                No per-iteration trace or action count is recorded; the iteration count
                                grows by the most passes any block ran (pieces any warp ran, with per-warp
                                scheduling, celer_set_async_warps). With a budget (celer_run_iterations) a
                                block stops after that many passes, or, per warp, the block drains once a
                                warp has run that many pieces: its queued tracks take their step without a
                                new step limit, so every track ends the run between two steps, as after a
                                synchronous iteration. Waits are bounded: if no track steps for about 1 s
                                the run ends with CELER_ERR_TIMEOUT or CELER_ERR_CAPACITY. */
};

/* Step until no track is alive or queued (Sec. 2: the outer loop over step
 * iterations, each applying the actions in turn to all active tracks and
 * refilling vacant slots from the initializer buffer; Sec. 3.4: all device
 * work and copies stay ordered on the context's stream), in one of the
 * CELER_LOOP_* modes. Synchronises the stream at the end. Returns
 * CELER_ERR_TIMEOUT at max_iterations, CELER_ERR_CAPACITY if the initializer
 * buffer is full and no track can make progress, CELER_ERR_INVALID for an
 * unknown mode or one the sort policy does not allow; the state stays
 * usable after each of these. */
celer_status celer_run_events(celer_ctx* ctx, int mode);

/* Profile of the persistent loop since creation, in SM cycles, n <= 10
 * entries: [0..3] time per phase as seen by the first block, barrier wait
 * included ([0] fill + step limit, [1] partition scatter, [2] along-step +
 * interactions, [3] unused); [4..7] sum over iterations of the slowest
 * block's work per phase; [8], [9] last-block bookkeeping after phases 0
 * and 2. */
celer_status celer_read_loop_profile(celer_ctx* ctx, uint64_t* cycles_out, int n);

/* As celer_run_events, but stop after at most `budget` more step iterations
 * (0: no limit); *done (nullable) receives the iterations run. A serving
 * loop uses this to return to the host between chunks of iterations, to
 * admit new events and collect finished ones while tracks stay resident.
 * In CELER_LOOP_ASYNC the budget counts each block's passes (or, with
 * per-warp scheduling, each warp's pieces, after which the block drains);
 * every track still ends the run between two steps. */
celer_status celer_run_iterations(celer_ctx* ctx, int mode, uint64_t budget, uint64_t* done);

/* Choose per-action launches (1) or per-phase launches (0) for the host and
 * graph loops. */
celer_status celer_set_split_actions(celer_ctx* ctx, int split);

/* Copy the energy-deposit tally of one event (n bins, n = the problem's bin
 * count) and its escaped energy into host memory: the detector hits that
 * Sec. 3.4 moves from device to host with a stream-ordered copy, per event
 * as in the mixed-event mode of Sec. 5.1. host_out: caller-owned, n doubles
 * (pageable or pinned); escaped: nullable. The copy is stream ordered and
 * the call then synchronises the context's stream only. n other than the
 * bin count: CELER_ERR_INVALID. */
celer_status celer_read_tallies(celer_ctx* ctx, uint32_t event, double* host_out, uint64_t n, double* escaped);

/* Zero the tally row, escaped energy and live-track count of an event so
 * that its row can be reused by a later event. */
celer_status celer_reset_event(celer_ctx* ctx, uint32_t event);

/* Number of live (alive or queued) tracks of an event; 0 once it is done. */
celer_status celer_event_live(celer_ctx* ctx, uint32_t event, uint64_t* live);

/* Per-primary records [first, first + count) in the order primaries were
 * added (history_capacity > 0): steps, secondaries, escaped and deposited
 * energy of each primary and all its descendants, the per-event results of
 * Sec. 5.1 resolved by primary, read out as in Sec. 3.4 (stream-ordered copy,
 * then the context's stream is synchronised). host_out: caller-owned, count
 * records; edep_out (nullable): count x n_bins deposits, row-major. A range
 * beyond the recorded primaries: CELER_ERR_INVALID. */
celer_status celer_read_history(celer_ctx* ctx, uint64_t first, uint64_t count, celer_history* host_out,
                                double* edep_out);

/* The problem the context was created with (pointer fields set to NULL). */
celer_status celer_get_problem(const celer_ctx* ctx, celer_problem* out);

/* Counters since creation (stream synchronised). */
celer_status celer_get_stats(celer_ctx* ctx, celer_step_stats* out);

/* Change the reordering policy between runs. */
celer_status celer_set_sort_policy(celer_ctx* ctx, int policy);

/* Per-iteration hit readout (Sec. 3.4, "Asynchronous memory management"):
 * during host-loop runs (CELER_LOOP_HOST), after every step iteration the
 * tally rows (max_events x bins doubles, row-major as in celer_read_tallies)
 * are copied into host_hits. mode 0: off. mode 1: stream-ordered
 * (cudaMemcpyAsync on the context's stream; other streams keep running).
 * mode 2: synchronous (the whole device is synchronised, then cudaMemcpy:
 * every stream waits for the copy, the behaviour the paper measured against).
 * host_hits: caller-owned, pinned (cudaHostAlloc or a pinned torch tensor) for
 * mode 1, at least max_events x bins doubles, valid while the mode is on.
 * Graph and persistent runs do not return to the host per iteration and copy
 * nothing. Bad mode, null or short buffer: CELER_ERR_INVALID. */
celer_status celer_set_hit_readout(celer_ctx* ctx, int mode, double* host_hits, uint64_t n);

/* Cap the GPU blocks of this context's kernels (0: the default, one block per
 * SM for the persistent and block-pass kernels), so that several contexts,
 * each on its own stream, can run their events side by side: the event-per-
 * stream mode the paper compares with one mixed track array (Sec. 4.1). The
 * next run starts with the new grids (a captured graph is rebuilt).
 * blocks < 0: CELER_ERR_INVALID. */
celer_status celer_set_grid_blocks(celer_ctx* ctx, int blocks);

/* Parent-slot reuse (Sec. 3.2, second paragraph): on = 1 makes the first of
 * the two photons of a pair conversion start in the slot of the photon that
 * converted, without passing through the initializer buffer; the second is
 * queued as before. Off by default. Histories do not change (a track's
 * history depends only on its initial state and id); the buffer traffic and
 * the fill work do. Takes effect at the next run. */
celer_status celer_set_parent_reuse(celer_ctx* ctx, int on);

/* Scheduling of the asynchronous loop (CELER_LOOP_ASYNC) for the block-local
 * policy. on = 0: block passes, as in the synchronous loops. on = 1: every
 * warp runs its own loop. It takes up to 32 tracks waiting for the same kind
 * of step (particle type and next action) from its block's queues in shared
 * memory, steps them, and queues the survivors again by their next kind. A
 * track then moves on as soon as its own step is done instead of waiting for
 * its block's slowest group. Charged tracks are taken before photons (their
 * steps form a shower's longest chains), and in runs without an iteration
 * budget all but the first two warps of a block take only full pieces of 32
 * (budgeted runs, such as a serving loop's chunks, let every warp take any
 * piece). A block holds at most 1024 live tracks in this
 * mode; a block that starts a run with more runs block passes. Histories do
 * not change. On by default. Takes effect at the next run. on outside
 * {0, 1}: CELER_ERR_INVALID. */
celer_status celer_set_async_warps(celer_ctx* ctx, int on);

/* Per-iteration counters (alive, queued, steps, tracks per action) of the
 * last min(n_max, recorded) iterations, the analogue of the paper's counter
 * tracks (Sec. 4). *n_out receives the row count. */
celer_status celer_read_trace(celer_ctx* ctx, celer_trace_row* host_out, uint64_t n_max, uint64_t* n_out);

/* Average device time per launch of each kernel over the last run, measured
 * with CUDA events when timing is enabled (enable != 0); names are static. */
celer_status celer_enable_kernel_timing(celer_ctx* ctx, int enable);
celer_status celer_kernel_timing(celer_ctx* ctx, const char** names, double* total_ms, uint64_t* launches,
                                 int n_max, int* n_out);

/* Stable partition of slot indices 0..n-1 by an 8-bit key, the same
 * partition the step loop builds (slots grouped by key in increasing key
 * order, ascending slot order within a key), as a stand-alone call that
 * allocates no device memory. The paper has no counterpart: this exists for
 * callers that cannot allocate device memory themselves, such as code that
 * runs while another framework's caching allocator owns the GPU memory, or a
 * host loop that cannot pay for cudaMalloc/cudaFree (cudaFree synchronises
 * the whole device).
 *
 * d_keys: n keys in device memory; keys not below n_keys are ignored (they
 * get no position). d_perm: device output; the slots of every key except
 * skip_key (-1: none) in partition order; positions of skip_key's slots and
 * positions from d_offsets[n_keys] on are left untouched. d_offsets: device
 * output of n_keys + 1 entries: d_offsets[k] is the first position of key k
 * and d_offsets[n_keys] the number of slots whose key is below n_keys (n
 * when every key is in range). The counts include skip_key's slots, which
 * occupy the last positions if skip_key is the largest key. n = 0 writes
 * zeros to d_offsets and nothing else (d_keys and d_perm may then be NULL).
 * Work is queued on cuda_stream (a cudaStream_t; NULL: the legacy default
 * stream); the call does not synchronise. If a CUDA error from earlier work
 * is pending on the calling thread, the call launches nothing, leaves that
 * error pending and returns CELER_ERR_CUDA.
 *
 * Working memory is one fixed array inside the library (256 KiB per device
 * that loads it, held until the process exits): n <= 2^20, n_keys <= 16,
 * otherwise CELER_ERR_INVALID. Every call on a device shares that array, so
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race and must be serialised by the caller. The first call on each device
 * looks up the array's device address with that device current; make that
 * first call before any stream capture. The address is kept for the life of
 * the process, so do not call this after cudaDeviceReset on that device. */
celer_status celer_partition_keys_noalloc(const uint8_t* d_keys, uint64_t n, int n_keys, int skip_key, uint32_t* d_perm,
                                          uint32_t* d_offsets, void* cuda_stream);

/* Live-track counts (alive or queued) of `count` consecutive tally rows
 * starting at first_row, into host memory. Synchronises the stream. */
celer_status celer_read_event_live(celer_ctx* ctx, uint32_t first_row, uint32_t count, uint32_t* host_out);

/* ---- serving: continuous batching of arriving events ---- */

typedef struct {
  double arrival_s;                 /* arrival time, seconds after the start of celer_serve */
  uint32_t event;                   /* event id (uses tally row event % max_events) */
  uint32_t pad;
  const celer_primary* primaries;   /* host */
  uint64_t n;
} celer_request;

typedef struct {
  double arrival_s;                 /* copied from the request */
  double admit_s;                   /* when its primaries were queued (-1: never) */
  double done_s;                    /* when its last track ended (-1: never) */
  double edep, escaped;             /* event totals, MeV */
} celer_request_result;

typedef struct {
  int mode;                         /* CELER_LOOP_* used for each chunk of iterations */
  uint64_t chunk_iterations;        /* iterations between host checks (0: 16) */
  double footprint_per_primary;     /* tracks reserved per primary at admission (0: 40) */
  uint32_t max_in_flight;           /* events on the device at once (0: no limit; 1: one at a time) */
  double stop_admitting_s;          /* no admission after this wall-clock time (0: serve every request);
                                       requests not admitted by then are left unserved */
  double* tallies_out;              /* nullable: n_requests x n_bins deposits, host */
} celer_serve_options;

typedef struct {
  double wall_s;                    /* from the start to the last completion */
  uint64_t track_steps;             /* track-steps taken during the call */
  uint64_t admitted, completed, chunks;
} celer_serve_summary;

/* Serve requests as they arrive (continuous batching, Sec. 5.1 "events mixed
 * in a single track array"): at each check the host admits, in arrival
 * order, every request that has arrived and whose expected footprint
 * (footprint_per_primary x primaries tracks) fits in the free part of the
 * slot store plus initializer buffer (slots + buffer entries, minus the
 * footprints of the events in flight) and whose tally row is free; then it
 * runs a chunk of step iterations with the tracks of all admitted events in
 * one slot array, and collects every event whose live-track count reached
 * zero (tallies copied to the host, row freed). Requests must be in
 * nondecreasing arrival order. Wall-clock times are measured on the host. */
celer_status celer_serve(celer_ctx* ctx, const celer_request* requests, uint64_t n, const celer_serve_options* options,
                         celer_request_result* results, celer_serve_summary* summary);

/* ---- autotuning of the launch configuration ---- */

typedef struct {
  uint64_t n_slots;
  int block_size, sort_policy, mode;
  double track_steps_per_s;         /* measured on the sample (0: the trial failed) */
  double ms;
  int async_warps;                  /* celer_set_async_warps of the trial (CELER_LOOP_ASYNC with the
                                       block-local policy is tried both ways; 1 elsewhere) */
} celer_tune_trial;

/* Try every combination of the given slot counts, block sizes, sort
 * policies and loop modes on a sample of primaries (grouped by their event
 * ids, events[i] for primaries[i]): a fresh context per combination, one
 * warm-up run, one timed run (CUDA events around celer_run_events). trials
 * (nullable, max_trials entries) receives every trial; best the fastest.
 * The base problem supplies everything else. CELER_LOOP_ASYNC pairs only
 * with the block-pass policies; other pairs are recorded with no
 * throughput. With the block-local policy it is tried with both of its
 * schedules (async_warps 1 and 0), so max_trials should allow for that
 * trial count. */
celer_status celer_autotune(const celer_problem* base, const celer_primary* primaries, const uint32_t* events,
                            uint64_t n, const uint64_t* slot_counts, int n_slot_counts, const int* block_sizes,
                            int n_block_sizes, const int* policies, int n_policies, const int* modes, int n_modes,
                            celer_tune_trial* trials, int max_trials, int* n_trials, celer_tune_trial* best);

/* ---- diagnostics used by the parity tests ---- */

/* Partition of the last iteration: per-slot key as used by the partition
 * (n_slots bytes; slots vacant at that time carry the last, vacant key), the permutation
 * (n_slots entries; the first offsets[n_keys - 1] are the live slots), the
 * n_keys + 1 offsets, and the number of blocks B that counted the keys.
 * Within a key the slots are ordered by the block owning their 32-slot chunk
 * (chunk c: block c mod B), then by chunk, then by slot. Valid only for the
 * sorted policies. */
celer_status celer_debug_partition(celer_ctx* ctx, uint8_t* keys_out, uint32_t* perm_out, uint32_t* offsets_out,
                                   int* n_keys, int* n_blocks);

/* Active-lane counters of the diagnostic build (compiled with
 * -DCELER_LANE_COUNTERS; the product build returns CELER_ERR_STATE). Sec. 3.1
 * judges reordering by the thread divergence it removes; these counters
 * measure it without a profiler. For each of the first min(n_max, 35) sites,
 * host_out receives three values: warp-level visits, the lanes active at
 * them summed (mean active lanes = lanes / visits), and the SM cycles spent
 * there summed where the site is timed (0 elsewhere). Sites: 0-7 the
 * per-warp pieces of the asynchronous loop by key (particle type and next
 * action, in the order photon boundary, electron boundary, electron range,
 * Compton, photoelectric, pair, Moller, brems; lanes = tracks claimed;
 * timed from the claim to the survivors' requeue), 8 its fills (timed), 9
 * the step limit, 10 the along-step, 11-15 the Compton, photoelectric, pair,
 * Moller and brems interactions, 16 and 17 one rejection attempt of the
 * Compton and Moller samplers, 18 the side-plane distance along the helix,
 * 19 the per-warp loop's rounds that found nothing to do (timed), 20-22 the
 * photon crossing pieces timed in three parts (choice and claim, the step,
 * the next step limit and requeue), 23-25 the same for electron crossings,
 * 26-30 a photon's step limit timed in five parts (state loads, grid position,
 * cross sections, distances to the planes, the rest with the stores), 31 the
 * per-warp loop's queueing of a track by its next kind, 32-34 the Compton
 * pieces timed in three parts as the crossings.
 * The counters cover every kernel launched since the last read on the
 * current device and are cleared by the read. *n_out receives the sites
 * written. Null pointers or n_max < 0: CELER_ERR_INVALID. */
celer_status celer_debug_lane_counts(uint64_t* host_out, int n_max, int* n_out);  /* 3 x n_max values */

/* Per-slot status (0 vacant, 1 alive, 2 waiting for buffer space) and
 * particle type (0 photon, 1 electron) into host arrays of n_slots bytes, and
 * the number of GPU blocks B of the block-pass policies (LOCAL, DATA): block b
 * owns the 32-slot chunks b, b + B, b + 2B, ... Checks the DATA policy's
 * charge partition of the fill (Sec. 3.2). */
celer_status celer_debug_slots(celer_ctx* ctx, uint8_t* status_out, uint8_t* ptype_out, int* n_blocks);

/* Per-slot track state into host arrays of n_slots entries: track id, event,
 * layer, and state_out = 7 x n_slots doubles, column-major (x, y, z, ux, uy,
 * uz, E; cm and MeV). Values of vacant slots are left over from their last
 * track (celer_debug_slots gives the status). For the kernel-level parity
 * test: one celer_step of primaries with given states against the oracle's
 * single step of each. Synchronises the context's stream. */
celer_status celer_debug_tracks(celer_ctx* ctx, uint64_t* tid_out, uint32_t* event_out, int32_t* layer_out,
                                double* state_out);

/* Check of the bounded waits of the persistent loops (no counterpart in the
 * paper): a cooperative launch of `blocks` (2-8) blocks meets at the loops'
 * grid barrier, which block `absent_block` never reaches (-1: every block
 * arrives, and the barrier must pass). The others must give
 * up after timeout_cycles SM cycles (at most 4e9), set the abort word and the
 * barrier-timeout error bit, and end. Returns CELER_ERR_TIMEOUT when they did
 * (error_bits and abort_word receive what the kernel left), CELER_OK if the
 * barrier passed, CELER_ERR_INVALID for bad arguments. Uses its own device
 * memory (allocated and freed here) and the legacy default stream. */
/* Check of the bounded queue waits of the asynchronous loop (no counterpart
 * in the paper): one thread waits for an entry to be written, either entry 0
 * of a one-entry initializer buffer (which = 0 or 2) or an entry of a
 * shared-memory queue of the per-warp schedule (which = 1 or 3). For
 * which = 0, 1 nothing writes the entry: the wait must give up after
 * timeout_cycles SM cycles (at most 4e9), set the abort word and the
 * timeout error bit, and end, and the call returns CELER_ERR_TIMEOUT
 * (error_bits and abort_word receive what the kernel left). For which = 2, 3
 * the entry was written first, the wait passes and the call returns
 * CELER_OK. CELER_ERR_INVALID for bad arguments. Uses its own device memory
 * (allocated and freed here) and the legacy default stream. */
celer_status celer_debug_queue_wait(int which, uint64_t timeout_cycles, uint32_t* error_bits, uint32_t* abort_word);

celer_status celer_debug_barrier_timeout(int blocks, int absent_block, uint64_t timeout_cycles, uint32_t* error_bits,
                                         uint32_t* abort_word);

/* Device table of material mat, column col (0 Compton, 1 photoelectric,
 * 2 pair, 3 Moller, 4 brems, 5 range), 200 values into host memory. */
celer_status celer_debug_table(celer_ctx* ctx, int mat, int col, double* host_out);

/* Run the device Philox4x32-10 on n (counter[4], key[2]) records (host,
 * 6 words each) and write the 4 output words of each into host_out. */
celer_status celer_debug_philox(const uint32_t* host_ctr_key, uint32_t* host_out, uint64_t n);

/* Same records through cuRAND's Philox4_32_10 device generator, mapped as
 * key = seed, counter = (0, 0, subsequence) + offset, for cross-checking. */
celer_status celer_debug_curand_philox(uint64_t seed, uint64_t subsequence, uint64_t offset4, uint32_t* host_out,
                                       uint64_t n);

/* Evaluate a binary64 function on n host arguments on the device: fn 0 the
 * table-driven logarithm of the step kernels, 1 their exponential, 4 and 5
 * their sin(2 pi x) and cos(2 pi x), 8 and 9 their sin(x) and cos(x) (helix
 * turns); 2, 3, 6, 7, 10, 11 CUDA's log, exp, sin(2 pi x), cos(2 pi x),
 * sin(x), cos(x) for comparison. No counterpart in the paper: it checks the
 * step kernels' elementary functions against the library's (accuracy about
 * 1 ulp). fn outside 0-11 or null pointers give CELER_ERR_INVALID. */
celer_status celer_debug_math(int fn, const double* host_x, uint64_t n, double* host_out);

/* Measure the device's FP64 throughput, the ceiling of the step kernels'
 * arithmetic: blocks_per_sm x (SM count) blocks of 256 threads each run 8
 * independent FP64 fused multiply-add chains for iters iterations, timed
 * with CUDA events after one shorter warm-up launch on the legacy default
 * stream. *tflops_out receives 2 x 8 x iters x threads / time in TFLOP/s,
 * *ms_out (nullable) the timed launch's duration. No counterpart in the
 * paper: it gives the measured peak beside the derived one. blocks_per_sm
 * outside 1-8, iters 0 or above 2^32, or a null tflops_out:
 * CELER_ERR_INVALID. Allocates and frees a small output buffer. */
celer_status celer_debug_fp64_rate(int blocks_per_sm, uint64_t iters, double* tflops_out, double* ms_out);

/* Draw one rejection sample per record on the device: which 0 the Compton
 * (Klein-Nishina, Butcher-Messel) sampler of the step kernels, which decides
 * each attempt in FP32 and falls back to FP64 near the acceptance boundary,
 * 1 its plain FP64 form, 2 the step kernels' Moller sampler (same FP32
 * filtering), 3 its plain FP64 form. Record i: energy host_E[i] MeV (photon
 * energy, or electron kinetic energy for Moller), random stream key
 * (seed, event), track id host_tid[i], draw counter host_ctr[i]; cut is the
 * Moller production cut (MeV, unused for Compton). Outputs (host arrays of n):
 * eps (E'/E, or T_delta/T), the Compton scattering cosine (0 for Moller), the
 * draw counter after sampling and the sampler's ok flag. No counterpart in
 * the paper: it checks that the filtered samplers give bit-identical results
 * to the plain FP64 ones. which outside 0-3 or null pointers give
 * CELER_ERR_INVALID. */
celer_status celer_debug_sample(int which, uint32_t seed, uint32_t event, const double* host_E, double cut,
                                const uint64_t* host_tid, const uint32_t* host_ctr, uint64_t n, double* eps_out,
                                double* cost_out, uint32_t* ctr_out, uint8_t* ok_out);

#ifdef __cplusplus
}
#endif
#endif
