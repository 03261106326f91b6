/*
 * hgp.h — C ABI of libhgp: GPU label-propagation refinement of a k-way hypergraph
 * partition under the connectivity (lambda-1) metric, for NVIDIA GB300 (sm_103a).
 *
 * The problem statement is the one of "Scalable Shared-Memory Hypergraph Partitioning"
 * (Gottesbüren, Heuer, Sanders, Schlag), Sec. 2: a weighted hypergraph H = (V, E, c, omega)
 * with positive weights, a k-way partition Pi : V -> {0..k-1} (the paper numbers blocks
 * 1..k), the balance bound L_max = (1+eps) * ceil(c(V)/k), the pin counts Phi(e, V_i), the
 * connectivity sets Lambda(e), and the objective (lambda-1)(Pi) = sum_e (lambda(e)-1) omega(e).
 * Refinement is the size-constrained label propagation of Sec. 6, with the gain
 * g_i(u) = b(u) - p_i(u) of Sec. 5, run in a deterministic synchronous form:
 *
 *   A round r is split into S sub-rounds.  Vertex u is active in sub-round
 *   splitmix64(seed ^ (r << 32 | u)) mod S (SplitMix64 output function).  It is eligible in
 *   the first round after creation (or after hgp_set_partition) and afterwards iff one of its
 *   incident nets had a pin moved in round r-1.  Every active eligible vertex picks the block
 *   with the highest positive gain whose weight, frozen at the start of the sub-round, plus
 *   c(u) is at most L_max; ties go to the smaller block id.  Candidates are approved per target
 *   block in (gain desc, vertex id asc) order while the inclusive prefix sum of their weights
 *   fits into L_max - w(t).  All approved moves are applied at once.
 *
 * All arithmetic is integer; results are bit-identical for any launch configuration and any
 * run.  Reading of the real-valued L_max: floor((1.0 + eps) * ceil(c(V)/k)) in IEEE double.
 * Empty nets contribute 0 to the objective.
 *
 * Conventions for every function:
 *   - Return value: an hgp_status (0 = success).  No function aborts, prints or exits.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA global memory of
 *     the current device.  Input arrays are owned by the caller and copied during the call;
 *     output arrays are owned by the caller.
 *   - A handle is used by one host thread at a time.  All device work is queued on the
 *     handle's stream (hgp_options.cuda_stream, or a stream the library creates); functions
 *     that return data to host memory synchronise that stream before returning.
 */
#ifndef HGP_H
#define HGP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HGP_OK = 0,
    HGP_ERR_INVALID = 1,      /* an argument or the hypergraph violates a stated rule */
    HGP_ERR_OOM = 2,          /* device or host allocation failed */
    HGP_ERR_UNSUPPORTED = 3,  /* k > 64, >= 2^31 pins, a vertex with sum of incident net
                                 weights >= 2^31, or more than 64 sub-rounds */
    HGP_ERR_CUDA = 4,         /* a CUDA call failed; the handle should be destroyed */
    HGP_ERR_TIMEOUT = 5,      /* a device-side wait gave up (batched persistent mode) */
    HGP_ERR_INTERNAL = 6      /* check mode found the maintained objective differing from
                                 the one recomputed from Phi */
} hgp_status;

typedef struct hgp_handle hgp_handle;
typedef struct hgp_batch hgp_batch;

/* Options.  Zero-initialised fields select the defaults given in brackets. */
typedef struct {
    int32_t subrounds;   /* S, 1..64 [4] */
    int32_t phi_width;   /* bytes per Phi entry: 1, 2 or 4; 0 = auto [0]: 1 if every net has
                            at most 255 pins, else 2.  Nets larger than the width can count
                            (255 or 65535 pins) keep 4-byte rows in a separate wide table. */
    uint64_t seed;       /* sub-round hash seed [0] */
    int32_t debug;       /* bit 0 (check mode): hgp_refine recomputes the objective from the
                            Phi table after the call and returns HGP_ERR_INTERNAL if it differs
                            from the incrementally maintained one; bit 1: build the vertex ->
                            nets lists with the bucketed transpose whatever the size (it is
                            otherwise used above 2^21 vertices); bit 2: store the nets in
                            internal order (by size class, largest first, so that the records
                            of the largest nets share L2 lines) whatever the size (it is
                            otherwise used from 2^20 nets on when the largest net has at least
                            8 times the average net size); bit 3: keep the input net order.
                            Results do not depend on the order; per-net outputs and
                            checkpoints always use input net ids; bit 4 (fault injection,
                            for tests of the error path): after each hgp_refine the maintained
                            objective is lowered by one from the host, so that check mode
                            reports HGP_ERR_INTERNAL [0] */
    int32_t graph;       /* 1: hgp_refine captures its launches as a CUDA graph on the first call
                            with a given round count and replays it afterwards [0]; ignored
                            while profiling is on */
    void *cuda_stream;   /* cudaStream_t to run on, or NULL for a library-owned stream */
    int32_t balance_moves;   /* variant (Sec. 6): a vertex without a feasible positive-gain
                                target may take a zero-gain move to a block t with room and
                                w(t) + c(u) < w(Pi(u)), the lightest such block [0] */
    int32_t revert_negative; /* variant (Sec. 5.2, Sec. 6): the attributed gain of each applied
                                move is its gain with every net seeing the sub-round's moves in
                                ascending vertex id (computed by Lemma 1, Sec. 5.4); after the
                                sub-round every move with a negative one is undone, and still
                                counts as a move for eligibility.  Adds a table of 32 * 2^ceil(
                                log2(2P)) bytes, n bytes and 4 m bytes.  Single handles only (a batch
                                rejects it) [0] */
    int32_t gain_ctas_per_sm;   /* persistent grid of the gain kernel, CTAs per SM; 0 = occupancy
                                   [0].  Results do not depend on it. */
    int32_t apply_ctas_per_sm;  /* the same for the apply kernel [0] */
} hgp_options;

/* Per-round statistics written by hgp_refine. */
typedef struct {
    int64_t objective;        /* (lambda-1)(Pi) after the round (Sec. 2) */
    int64_t candidates;       /* vertices that chose a target in the round */
    int64_t approved;         /* moves applied in the round */
    int64_t eligible;         /* eligible vertices in the round */
    int64_t max_block_weight; /* max_i c(V_i) after the round */
    int64_t moved_pins;       /* sum of d(u) over the vertices moved in the round */
    int64_t reverted;         /* moves undone by the revert variant in the round */
} hgp_round_stats;

/* Device time per phase of the rounds, from CUDA events recorded on the handle's stream
 * around each kernel while profiling is on (hgp_set_profiling).  Phases: 0 sub-round lists,
 * 1 gain and best target, 2 approval, 3 apply (Phi, Lambda, objective), 4 end of round,
 * 5 attributed gains and reverts (revert variant only). */
#define HGP_PHASES 6
typedef struct {
    double ms[HGP_PHASES];         /* accumulated milliseconds */
    int64_t launches[HGP_PHASES];  /* kernel launches accumulated into ms[] */
} hgp_profile;

/* Fills *opt with the defaults. */
void hgp_default_options(hgp_options *opt);

/* Human-readable name of a status code (static string). */
const char *hgp_strerror(int code);

/*
 * Creates a handle from a hypergraph in net->pins CSR form (paper Sec. 2 notation;
 * Sec. 3.2 describes the same adjacency arrays), copying all inputs to the device.
 *
 *   n, m          number of vertices and nets, n >= 1, m >= 0.
 *   net_offsets   host int64[m+1]: pins of net e are pins[net_offsets[e] .. net_offsets[e+1]);
 *                 net_offsets[0] = 0, non-decreasing, net_offsets[m] = P < 2^31.
 *   pins          host int32[P]: vertex ids in [0, n), strictly increasing within each net.
 *   vertex_w      host int32[n] with every c(v) >= 1, or NULL for unit weights.
 *   net_w         host int32[m] with every omega(e) >= 1, or NULL for unit weights.
 *   k             number of blocks, 2..64.   eps: balance parameter, 0 < eps < 1 (Sec. 2).
 *   initial_part  host int32[n] with values in [0, k); need not be balanced.
 *   opt           NULL for defaults.
 *   out           receives the handle; set to NULL on any error (nothing leaks).
 * Errors: HGP_ERR_INVALID for any violated rule above or null required pointers;
 * HGP_ERR_UNSUPPORTED for k > 64, P >= 2^31, S > 64, or a vertex whose incident net weights
 * sum to 2^31 or more; HGP_ERR_OOM; HGP_ERR_CUDA.
 */
int hgp_create(int32_t n, int32_t m, const int64_t *net_offsets, const int32_t *pins,
               const int32_t *vertex_w, const int32_t *net_w, int32_t k, double eps,
               const int32_t *initial_part, const hgp_options *opt, hgp_handle **out);

/* Same as hgp_create, but every array argument is a DEVICE pointer (copied device to
 * device; the caller may free its buffers after the call returns). */
int hgp_create_device(int32_t n, int32_t m, const int64_t *net_offsets, const int32_t *pins,
                      const int32_t *vertex_w, const int32_t *net_w, int32_t k, double eps,
                      const int32_t *initial_part, const hgp_options *opt, hgp_handle **out);

/*
 * Runs `rounds` (>= 0) synchronous label-propagation rounds (Sec. 6) on the handle's stream.
 * stats: NULL, or host hgp_round_stats[rounds] filled on return (the call then synchronises).
 * With stats == NULL the call returns after queuing the work; a later call that returns data
 * synchronises.  Round numbering and eligibility continue across calls, so refine(a) followed
 * by refine(b) equals refine(a+b).
 */
int hgp_refine(hgp_handle *h, int32_t rounds, hgp_round_stats *stats);

/* Replaces the partition (host int32[n], or DEVICE pointer if on_device != 0), rebuilds Phi,
 * Lambda, block weights and the objective, and restarts round numbering at 0 with every
 * vertex eligible, exactly as if the handle had been created with this partition. */
int hgp_set_partition(hgp_handle *h, const int32_t *part, int32_t on_device);

/*
 * Checkpoint / resume.  Everything later rounds depend on: the partition (int32[n]), which nets
 * had a pin moved in the last completed round (uint8[m], 1 = moved; these decide eligibility in
 * the next round, Sec. 6), the next round number (it selects the sub-rounds), and whether the
 * next round is the first one after creation (every vertex eligible).  All arrays are host
 * memory.  hgp_import_state on a handle created from the same hypergraph and options continues
 * exactly where the exported handle stopped: refine(a); export; import; refine(b) equals
 * refine(a + b).  moved_nets may be NULL on import only when first_round != 0.
 */
int hgp_export_state(hgp_handle *h, int32_t *part, uint8_t *moved_nets, int64_t *next_round,
                     int32_t *first_round);
int hgp_import_state(hgp_handle *h, const int32_t *part, const uint8_t *moved_nets,
                     int64_t next_round, int32_t first_round);

/* (lambda-1)(Pi) as maintained incrementally (Sec. 2). */
int hgp_objective(hgp_handle *h, int64_t *out);

/* (lambda-1)(Pi) recomputed from scratch from the Phi table (check mode). */
int hgp_objective_from_phi(hgp_handle *h, int64_t *out);

/* Current partition into host int32[n] (or a device pointer with on_device != 0). */
int hgp_get_partition(hgp_handle *h, int32_t *part, int32_t on_device);

/* Block weights c(V_i) into host int64[k]. */
int hgp_get_block_weights(hgp_handle *h, int64_t *w);

/* Phi(e, V_i) widened to host int32[m*k], row-major by net in input order (Sec. 5.1). */
int hgp_get_phi(hgp_handle *h, int32_t *phi);

/* Connectivity sets Lambda(e) as host uint64[m] bitsets (bit i = block i). */
int hgp_get_lambda(hgp_handle *h, uint64_t *lam);

/* Sizes and derived constants: n, m, k, P, L_max, Phi width in bytes, number of wide nets,
 * next round number.  Any pointer may be NULL. */
int hgp_get_info(hgp_handle *h, int32_t *n, int32_t *m, int32_t *k, int64_t *pins,
                 int64_t *lmax, int32_t *phi_width, int32_t *wide_nets, int64_t *next_round);

/*
 * Debug export of the gain step alone: computes, against the current state, the candidates of
 * sub-round s (0 <= s < S) of the next round, without applying anything.  target: host
 * int32[n] (-1 for vertices that are inactive, ineligible or without a feasible positive-gain
 * block); gain: host int64[n] (0 where target is -1).
 */
int hgp_debug_candidates(hgp_handle *h, int32_t s, int32_t *target, int64_t *gain);

/*
 * Batches: many handles (hypergraphs of uneven sizes, any k and Phi width) refined together.
 * Every phase of a round is one kernel launch over the work items of all member handles
 * (members with k <= 32 and k > 32 form two groups), and by default the launches of a
 * hgp_batch_refine call are captured once as a CUDA graph and replayed.  The arithmetic of
 * each member is unchanged: refining a handle inside a batch gives exactly the result of
 * refining it alone.  The batch does not own the handles: they must not be used elsewhere while
 * a batch call runs, and their round numbering advances with the batch.  A member may be
 * destroyed before the batch only if the batch is then used for nothing but hgp_batch_destroy.
 */
typedef struct {
    int32_t graph;              /* 1: capture/replay a CUDA graph per round count [1] */
    int32_t gain_ctas_per_sm;   /* persistent grid of the gain kernel, CTAs per SM; 0 = occupancy */
    int32_t apply_ctas_per_sm;  /* persistent grid of the apply kernel, CTAs per SM; 0 = occupancy */
    int32_t reserved;
    void *cuda_stream;          /* stream the batch runs on, or NULL for a library-owned stream */
} hgp_batch_options;

void hgp_batch_default_options(hgp_batch_options *opt);

/* handles: host array of `count` distinct handles on the current device.  Returns
 * HGP_ERR_UNSUPPORTED for a handle created with the revert variant.  Members may live on other
 * streams than the batch: every hgp_batch_refine call then starts, on the device, after the
 * work already queued on those streams, and work queued on them afterwards (read-backs,
 * hgp_destroy) runs after the call; no call blocks the host for this.  A handle may be a member
 * of several batches on different streams: a call also starts after the last call of another
 * batch that refined one of its members. */
int hgp_batch_create(hgp_handle *const *handles, int32_t count, const hgp_batch_options *opt,
                     hgp_batch **out);

/* Runs `rounds` rounds on every member.  stats: NULL or host hgp_round_stats[count * rounds],
 * member-major (member i's rounds at [i * rounds, (i + 1) * rounds)); filled on return, and the
 * call then synchronises.  Without stats the call returns with the work queued. */
int hgp_batch_refine(hgp_batch *b, int32_t rounds, hgp_round_stats *stats);

/* Statistics of the last hgp_batch_refine call, laid out as that call's `stats` argument;
 * `rounds` must equal that call's round count (else HGP_ERR_INVALID).  Waits for that call
 * only, not for work queued on the batch's stream after it.  Lets a caller queue a call without
 * statistics, do host work (and queue further work, for example the next call of another
 * batch) while it runs, and read them afterwards. */
int hgp_batch_get_stats(hgp_batch *b, int32_t rounds, hgp_round_stats *stats);

/* done: 1 if the last hgp_batch_refine call has finished on the device (or there was none),
 * else 0.  Does not block. */
int hgp_batch_query(hgp_batch *b, int32_t *done);

/* Partitions Pi of the members listed in `members` (count indices into the batch's handles) as
 * they are after the batch's last hgp_batch_refine call, written back to back into host int32
 * `out` (the members' vertex counts summed, in the listed order).  Waits for that call only;
 * one copy and one wait for all of them (a serving loop retiring the members a call finished).
 * The copy goes through one page-locked staging buffer of the library (grown when a call needs
 * more, kept for the life of the process), so concurrent calls run one after another.
 * HGP_ERR_INVALID for a null batch, a negative count, null arrays with count > 0, or an index
 * outside [0, members of the batch). */
int hgp_batch_get_partitions(hgp_batch *b, const int32_t *members, int32_t count, int32_t *out);

/* Waits for the batch's queued work. */
int hgp_batch_synchronize(hgp_batch *b);

/* Kernel launches issued by the batch so far (graph replays count their kernels). */
int hgp_batch_get_launch_count(hgp_batch *b, int64_t *out);

void hgp_batch_destroy(hgp_batch *b);

/* Turns per-phase event timing on (enable != 0) or off, and clears the accumulated profile.
 * While on, hgp_refine synchronises the handle's stream before returning. */
int hgp_set_profiling(hgp_handle *h, int32_t enable);

/* Profile accumulated since profiling was last enabled. */
int hgp_get_profile(hgp_handle *h, hgp_profile *out);

/* Number of kernels the handle has launched since creation (all phases, setup included). */
int hgp_get_launch_count(hgp_handle *h, int64_t *out);

/*
 * Allocation-free gain step.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory when they need the computation, for example
 * code running while an application allocator owns the whole device, inside host callbacks
 * where cudaMalloc is not allowed, or on latency-critical paths that must not block on the
 * allocator.  It calls no cudaMalloc, cudaFree or allocating library routine.
 *
 * Computes, for the partition `part`, the candidates of sub-round s (0 <= s < subrounds) of
 * the first round (every vertex eligible), exactly as hgp_debug_candidates does on a handle
 * freshly created from the same inputs and options: target[u] = best block or -1, gain[u] =
 * its gain or 0.
 *
 *   All arrays are DEVICE pointers owned by the caller: net_offsets int32[m+1] and pins
 *   int32[P] (net -> pins, pins strictly increasing inside each net), vtx_offsets int32[n+1]
 *   and inc_nets int32[P] (vertex -> incident nets, the transpose of the first CSR: vertex v
 *   lists exactly the nets that have v as a pin, in increasing net id), vertex_w int32[n] /
 *   net_w int32[m] or NULL for unit weights, part int32[n]; outputs target int32[n] and gain
 *   int64[n].  Work is queued on cuda_stream (NULL = default stream); the call synchronises
 *   that stream to validate the inputs, then returns with the computation queued.  It must
 *   not be called while that stream is being captured (it then returns HGP_ERR_INVALID).
 *   Limit: m <= 262144 nets (2^18); k <= 64; subrounds <= 64.  Larger m returns
 *   HGP_ERR_UNSUPPORTED.  Out-of-range offsets, pins, incident nets, partition entries,
 *   non-positive weights, unsorted or repeated pins or nets, and a vertex -> nets CSR that is
 *   not the transpose of the net -> pins CSR return HGP_ERR_INVALID before the computation
 *   runs.
 *   Scratch: a fixed 8 MiB device array inside the library, held on every GPU that loads the
 *   library until the process exits.  Its address is looked up on the first call made on
 *   each device (with that device current), so that first call should come before any
 *   stream capture.  All calls share the array and it keeps the last call's contents:
 *   calls whose work overlaps on the GPU race and must be serialised by the caller.
 */
int hgp_candidates_noalloc(int32_t n, int32_t m, const int32_t *net_offsets, const int32_t *pins,
                           const int32_t *vtx_offsets, const int32_t *inc_nets,
                           const int32_t *vertex_w, const int32_t *net_w, int32_t k, double eps,
                           const int32_t *part, int32_t subrounds, uint64_t seed, int32_t s,
                           int32_t *target, int64_t *gain, void *cuda_stream);

/*
 * Sets the persistent grids of the handle's gain and apply kernels (CTAs per SM; 0 = derived
 * from occupancy), as the options of the same names do at creation.  Results never depend on
 * them.  Waits for the handle's stream; drops a captured CUDA graph.
 */
int hgp_set_launch_shape(hgp_handle *h, int32_t gain_ctas_per_sm, int32_t apply_ctas_per_sm);

/*
 * Rebalancing (paper Sec. 8), in a synchronous form.  Runs passes while a block is heavier
 * than L_max, at most max_passes.  A pass splits the vertices into the handle's S sub-rounds
 * (hash round number 2^30 + pass index).  In a sub-round, against the state at its start,
 * every vertex u of an overloaded block a picks the block t != a with room (w(t) + c(u) <=
 * L_max) of highest gain (smaller id on ties).  The first pass is phase 1, which keeps only
 * gains >= 0 (the paper's one sweep of immediate non-negative moves); later passes are phase
 * 2, which keeps any gain (least connectivity increase first).  Candidates are ordered by
 * (gain desc, id asc); per
 * source block, a candidate passes while the weight that left before it is below
 * w(a) - L_max; per target block, passing candidates are approved while their inclusive
 * prefix fits L_max - w(t).  A phase-2 pass without moves ends the call.  Rebalancing moves
 * do not count as moves for LP eligibility and do not advance the round number.
 * stats: NULL or host hgp_round_stats[max_passes]; entry i describes pass i (eligible =
 * vertices of overloaded blocks considered, reverted = 0).  phases: NULL or host
 * int32[max_passes] (1 or 2).  num_passes: NULL or receives the number of passes run.
 * HGP_ERR_UNSUPPORTED when twice the largest incident net weight of a vertex reaches 2^31.
 */
int hgp_rebalance(hgp_handle *h, int32_t max_passes, hgp_round_stats *stats, int32_t *phases,
                  int32_t *num_passes);

/*
 * Contraction (paper Sec. 3.2): the coarse hypergraph of a vertex clustering.
 * Inputs are DEVICE arrays (as for hgp_create_device): net_off int64[m+1], pins int32[P]
 * (P = net_off[m] < 2^31), vertex_w / net_w int32 or NULL (unit), cluster int32[n] with values
 * in [0, n).  Cluster ids are remapped to 0..n'-1 in increasing order; the coarse weight of a
 * cluster is the sum of its vertex weights; every net's pins are mapped to their clusters,
 * sorted and de-duplicated; nets left with fewer than two pins are dropped; identical nets
 * (equal sorted pin lists) become one net whose weight is the sum of theirs, at the position
 * of the smallest original net id, and the coarse nets keep the order of those nets.
 * Runs on cuda_stream (NULL: the legacy default stream) and synchronises it; on success *out
 * owns the coarse arrays on the current device (release with hgp_coarse_destroy).
 * HGP_ERR_INVALID for a cluster id out of range; HGP_ERR_UNSUPPORTED when a coarse vertex or
 * net weight reaches 2^31 or P >= 2^31.  The coarse arrays are valid inputs of
 * hgp_create_device (pins strictly increasing inside each net).
 */
typedef struct hgp_coarse hgp_coarse;
int hgp_contract(int32_t n, int32_t m, const int64_t *net_off, const int32_t *pins,
                 const int32_t *vertex_w, const int32_t *net_w, const int32_t *cluster,
                 void *cuda_stream, hgp_coarse **out);
/* n', m' and P' of the coarse hypergraph. */
int hgp_coarse_get_sizes(const hgp_coarse *c, int32_t *n, int32_t *m, int64_t *num_pins);
/* Device pointers owned by c (any may be NULL): net_off int64[m'+1], pins int32[P'],
 * vertex_w int32[n'], net_w int32[m'], map int32[n] (coarse id of every fine vertex). */
int hgp_coarse_get_device_arrays(const hgp_coarse *c, const int64_t **net_off, const int32_t **pins,
                                 const int32_t **vertex_w, const int32_t **net_w, const int32_t **map);
/* Copies the coarse arrays to host buffers of the sizes above (any may be NULL). */
int hgp_coarse_copy_to_host(const hgp_coarse *c, int64_t *net_off, int32_t *pins, int32_t *vertex_w,
                            int32_t *net_w, int32_t *map);
/* fine_part[u] = coarse_part[map[u]] (device int32 arrays of n' and n entries). */
int hgp_coarse_project(const hgp_coarse *c, const int32_t *coarse_part, int32_t *fine_part);
void hgp_coarse_destroy(hgp_coarse *c);

/*
 * Exact gains of a move sequence (paper Sec. 5.4, Lemma 1), computed in parallel.
 * moves: host int32[count][3] = (u, from, to) in sequence order, every vertex at most once,
 * from = its current block, to != from.  gains: host int64[count], gains[j] = the gain (Sec. 5)
 * of move j against the state after moves 0..j-1 were performed.  The handle's partition is
 * not changed.  HGP_ERR_INVALID for an invalid move or sequence.
 */
int hgp_exact_gains(hgp_handle *h, int32_t count, const int32_t *moves, int64_t *gains);

/*
 * Measurement helper (no counterpart in the paper): times n_gathers random 32-byte gathers from
 * a freshly allocated array of array_bytes bytes on the current device (best of two timed runs
 * after one warm-up) and returns the time and the rate.  The gain and apply steps are bound by
 * such random accesses, so this rate is their ceiling when the per-net data exceeds L2.
 * Allocates and frees its own buffers.
 */
int hgp_probe_gather(int64_t array_bytes, int64_t n_gathers, double *ms_out, double *gathers_per_s);

/*
 * Measurement helper (no counterpart in the paper): times n_atomics 32-bit atomic additions,
 * each at a random word of a freshly allocated array of array_bytes bytes and each returning
 * the old value that the thread then uses (the form of the apply step's pin-count updates), and
 * returns the time and the rate.  Allocates and frees its own buffers.
 */
int hgp_probe_atomic(int64_t array_bytes, int64_t n_atomics, double *ms_out, double *atomics_per_s);

/* Frees all device memory of the handle (NULL is allowed).  The releases are queued on the
 * handle's stream behind its pending work, so the call returns without waiting for the device;
 * the memory returns to the library's pool (see hgp_set_pool_retention). */
void hgp_destroy(hgp_handle *h);

/*
 * Memory pool (no counterpart in the paper).  Handles and batches take their device memory
 * from a stream-ordered pool the library keeps per device (allocations and releases are
 * queued on the owner's stream and never synchronise the device, so handles can be created
 * and destroyed while other handles' kernels run).  By default freed memory goes back to the
 * system at the next synchronisation; this call lets the pool of the current device keep up
 * to `bytes` of freed memory for reuse, which a caller that creates and destroys many
 * handles (a serving loop) may want.  HGP_ERR_INVALID for bytes < 0.
 */
int hgp_set_pool_retention(int64_t bytes);

/* Host waits inside the library (read-backs, the end of hgp_create, statistics): on = 0
 * (default) spins in cudaStreamSynchronize; on = 1 sleeps on a blocking-sync event recorded on
 * the stream, which frees the CPU core while the device works (for callers where many threads
 * wait at once, such as a serving loop's creator threads) at the cost of a wake-up latency.
 * Process-wide; results do not depend on it. */
int hgp_set_blocking_waits(int32_t on);

#ifdef __cplusplus
}
#endif
#endif /* HGP_H */
