/*
 * gx -- breadth-first exploration of a network of synchronising LTSs on one
 * GB300 GPU, with a warp-cooperative bucketed find-or-put hash table.
 *
 * The method is the one of "On the Scalability of the GPUexplore
 * Explicit-State Model Checker" (Cassee, Neele, Wijs): a network of labelled
 * transition systems (Sec. 3, Fig. 1) is explored level by level; every
 * successor goes through a find-or-put on a closed-hashing table whose
 * buckets are read by a group of cooperating threads and claimed by
 * compare-and-swap, with a new bucket picked by the next hash-constant set
 * when a bucket is full (Sec. 4.1, Figs. 3-4); the bucket size is
 * configurable from 32 words down to 4 (Sec. 4.2, Fig. 5).
 *
 * Conventions for every entry point:
 *   - Return value: a gx_status.  On failure gx_last_error() gives a
 *     human-readable message (thread-local, valid until the next call on the
 *     same thread).  No entry point aborts or traps.
 *   - "device pointer" arguments must point to memory of the current CUDA
 *     device; "host pointer" arguments to ordinary (or pinned) host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device work is issued on it; calls that return host-visible
 *     results synchronise that stream before returning.
 *   - Input arrays are owned by the caller and are only read during the call.
 *   - Threads: calls on different gx_net / gx_batch handles may run
 *     concurrently; calls on the same handle must not (a handle keeps the
 *     last search's results and its cached CUDA graphs).
 */
#ifndef GX_H
#define GX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gx_status {
  GX_OK = 0,
  GX_ERR_INVALID = 1,            /* bad argument or network (message says which) */
  GX_ERR_OOM = 2,                /* workspace too small / device allocation failed */
  GX_ERR_TABLE_FULL = 3,         /* every hash-constant set met a full bucket (Sec. 4.1) */
  GX_ERR_FRONTIER_OVERFLOW = 4,  /* the frontier ring could not hold the next level */
  GX_ERR_SPIN_LIMIT = 5,         /* a bounded device wait gave up */
  GX_ERR_CUDA = 6,               /* a CUDA runtime call failed */
  GX_ERR_STATE = 7               /* call order (e.g. stats before any exploration) */
} gx_status;

/* ------------------------------------------------------------------------------------------
 * Networks (Sec. 3, Fig. 1).
 *
 * A process is an LTS: n_states local states numbered 0..n_states-1, an
 * initial state and n_edges labelled edges (src[i] -label[i]-> dst[i]).
 * Labels are global ids 0..n_labels-1.  A rule is a synchronisation vector:
 * its n_parts participants (proc[j], label[j]) -- distinct processes -- move
 * together when each has an edge with its label from its current state; every
 * combination of such edges is one transition.  A (process, label) pair that
 * occurs in any rule never moves alone; every other edge moves its process
 * alone (interleaving).  result_label is kept for reference only.
 * ---------------------------------------------------------------------------------------- */
typedef struct gx_lts {
  uint32_t n_states, n_edges, initial;
  const uint32_t *src, *label, *dst; /* host pointers, n_edges each */
} gx_lts;

typedef struct gx_rule {
  uint32_t n_parts;
  const uint32_t *proc, *label; /* host pointers, n_parts each */
  uint32_t result_label;
} gx_rule;

typedef struct gx_net_desc {
  uint32_t n_procs, n_labels;
  const gx_lts* procs;   /* host pointer, n_procs entries */
  uint32_t n_rules;
  const gx_rule* rules;  /* host pointer, n_rules entries (may be NULL if 0) */
} gx_net_desc;

typedef struct gx_net gx_net; /* opaque, owned by the library; free with gx_free */

/* Validate and encode a network (Sec. 3 network of LTSs; bit-packed 32-bit
 * state vectors as in Sec. 3 and Sec. 4.2, "the vector size generally does
 * not exceed four integers").  Each process gets ceil(log2 n_states) bits
 * (at least 1); fields are packed LSB-first into 32-bit words whose bit 31
 * is reserved (always set in a stored vector, so an all-zero slot is empty);
 * a field never straddles two words.  At most 4 words (3 are padded to 4).
 * Errors: GX_ERR_INVALID for out-of-range states/labels/processes, repeated
 * processes in one rule, empty rules, rules of more than 16 processes, more
 * than 124 processes, vectors longer than 4 words, or an upper bound of 2^32
 * or more on one state's successors (the sum over processes of their most
 * local edges from one state, plus over rules of the product of their
 * participants' most matching edges from one state).
 * Host-only: no device memory is touched.  *out is set only on GX_OK. */
gx_status gx_load_network(const gx_net_desc* desc, gx_net** out);

/* Release a network and everything the library holds for it.  NULL is a no-op. */
void gx_free(gx_net* net);

/* A network in the paper's input format (Sec. 3, Fig. 1): an EXP.OPEN
 * composition
 *     par using v_1, ..., v_m in "f_1" || ... || "f_n" end par
 * ("using v_1, ..., v_m" may be left out), where each synchronisation vector
 * v_j is  l_1 * ... * l_n -> r : one label per process, or '_' for a process
 * that does not take part, and the result label r.  Each "f_i" names an LTS
 * given in Aldebaran format:
 *     des (initial, n_transitions, n_states)
 *     (src, "label", dst)        one line per transition
 * Labels are global strings (quotes optional where a label has no comma,
 * quote or parenthesis); a (process, label) pair occurring in some vector
 * moves only through vectors, every other transition interleaves.
 * Comments (* ... *) may appear in the composition.
 * exp_text: the composition; file_names / file_texts: n_files names (as
 * written between the quotes) and contents, host memory, copied.  Several
 * processes may name the same file.  On success *out is a network as from
 * gx_load_network, with label names for gx_label_name.  GX_ERR_INVALID with a
 * message naming the file and line on a syntax error, a vector whose length
 * differs from the number of processes, a file not given, a state out of
 * range or a transition count that does not match the des header. */
gx_status gx_load_exp(const char* exp_text, uint32_t n_files, const char* const* file_names,
                      const char* const* file_texts, gx_net** out);

/* Name of label `label` of a network from gx_load_exp (the decimal index for
 * networks from gx_load_network), NUL-terminated into buf (cap bytes,
 * truncated); *len gets the full length. */
gx_status gx_label_name(const gx_net* net, uint32_t label, char* buf, uint32_t cap, uint32_t* len);

/* Sizes of a loaded network: processes, labels, synchronisation rules and
 * transitions over all process LTSs.  Any output may be NULL. */
gx_status gx_network_counts(const gx_net* net, uint32_t* n_procs, uint32_t* n_labels, uint32_t* n_rules,
                            uint64_t* n_edges);

/* Message of the last failing call on this thread ("" if none). */
const char* gx_last_error(void);

/* Vector layout chosen by gx_load_network: words per vector (1, 2 or 4 after
 * padding) and, per process, the word index, bit offset and bit width of its
 * field (each array n_procs long; any of them may be NULL). */
gx_status gx_layout(const gx_net* net, uint32_t* vector_words, uint32_t* field_word,
                    uint32_t* field_offset, uint32_t* field_bits);

/* ------------------------------------------------------------------------------------------
 * Exploration options.
 * ---------------------------------------------------------------------------------------- */
typedef struct gx_explore_opts {
  uint32_t bucket_words;   /* B, words per bucket: 4, 8, 16 or 32 (Sec. 4.2).  0 = 8 */
  uint32_t group_lanes;    /* G, threads sharing one bucket: a power of two with
                              1 <= G <= B / vector_words.  0 = B / vector_words
                              (one thread per slot) */
  uint32_t hash_rounds;    /* hash-constant sets tried per insertion, 1..64.
                              0 = 8 (Sec. 4.1) */
  uint32_t stop_at_first_deadlock; /* finish the level that met the first deadlock, then stop */
  uint32_t max_levels;     /* stop after this many levels have been expanded; 0 = no limit */
  uint32_t deadlock_cap;   /* deadlock states kept for gx_deadlocks; 0 = 1024 */
  uint32_t ctas_per_sm;    /* persistent CTAs per SM; 0 = as many as fit */
  uint32_t guided_batch;   /* GX_DL_GUIDED: open states expanded per iteration; 0 = 8192 */
  uint64_t table_bytes;    /* hash-table size; rounded down to a power-of-two number of
                              buckets.  0 = 1 GiB */
  uint64_t frontier_states;/* capacity of the frontier ring in vectors; rounded up to a
                              power of two.  0 = table slots / 4 (at least 4096) */
  /* Partitioned expansion (a slice-ordered form of the paper's batched flush of
   * new vectors into the table, Sec. 3): a level's successors are counted per
   * table slice, written slice by slice into a buffer and then looked up slice
   * by slice, so the part of the table being probed stays in L2.  Off by
   * default: on the networks measured so far the direct path is faster. */
  uint64_t successor_buffer;     /* buffer capacity in vectors (< 2^32); 0 = table slots / 2 */
  uint32_t slice_log2;           /* 2^slice_log2 table slices; 0 = auto (about 32 MiB each,
                                    at most 4096 slices) */
  uint32_t partition_min_states; /* levels with at least this many states are partitioned;
                                    0 = never (default) */
  uint32_t guided_bins;          /* GX_DL_GUIDED: priority bins; 0 = 32 */
  uint32_t warp_cache_log2;      /* per-warp cache of recently seen vectors (the block-local
                                    state cache of Fig. 2): 2^n entries per warp in shared
                                    memory (2^(n-1) for 4-word vectors, the same bytes), a hit
                                    skips find-or-put.  0 = off, 1..12 = 2^n, 0xFFFFFFFF =
                                    automatic (gx_default_opts): 2^9 unless the GPU-wide
                                    cache below is in use (together they measured slower);
                                    2^6 with the queued 4-word kernel (region_passes), whose
                                    CTAs then still fit 5 per SM */
  float guided_scale;            /* GX_DL_GUIDED: score at which a state falls in the last
                                    bin (scores are predicted distances / max_dist); 0 = 1.0 */
  uint32_t watch;                /* 1 = safety check (Sec. 3: the negation of a safety property
                                    is added to the network as one more automaton): an explored
                                    state whose process watch_proc is in local state watch_state
                                    (the automaton's error state) is a violation.  BFS searches
                                    only (gx_explore, GX_DL_BFS_*) */
  uint32_t watch_proc, watch_state;
  uint32_t stop_at_first_violation; /* 1 = stop after the level holding the first violation
                                    (every violation of that level is reported) */
  uint32_t violation_cap;        /* violating states kept for gx_violations; 0 = 1024 */
  uint32_t host_loop;            /* 1 = drive the level loop from the host (one control-block
                                    read per level, per-level CUDA-event times).  0 (default):
                                    when the partitioned path is off, the levels run on the
                                    device as one CUDA graph with a conditional WHILE node
                                    (expand, then a one-thread advance step that records the
                                    level and decides whether to go on); after 4096 levels the
                                    host loop takes over */
  uint32_t region_passes;        /* passes per BFS level of the direct path, a power of two
                                    1..16: pass q probes only the successors whose first
                                    bucket lies in region q of the table (its q-th
                                    1/region_passes of the buckets); every pass generates
                                    all successors of the level, the first one counts them.
                                    One pass's random table reads then stay inside one
                                    region: on GB300 random reads run at the full rate
                                    within any 64 GiB and 4x slower across 128 GiB
                                    (address-translation reach).  In a table above 64 GiB
                                    every hash round of a vector stays inside the 64 GiB
                                    span of its first bucket, so later rounds stay in the
                                    pass's region too.  With more than one pass, 4-word
                                    slots in 4- or 8-word buckets with one lane per bucket
                                    run the level kernel with the successor queue (only the
                                    pass's successors are probed, 32 at a time).  Results
                                    do not depend on it.  0 = auto: the fewest passes whose
                                    regions are at most 64 GiB (1 for tables up to 64 GiB) */
  uint32_t global_cache_log2;    /* GPU-wide cache of recently seen vectors: 2^n
                                    direct-mapped 64-bit entries in the workspace, cleared at
                                    the start of each search and small enough to stay in L2.
                                    An entry holds a vector exactly: 1- and 2-word vectors
                                    as they are, 4-word vectors as their field bits packed
                                    into 64 (no effect on 4-word vectors whose fields take
                                    more than 64 bits).  A vector goes in after its
                                    find-or-put found or inserted it, so a hit is a known
                                    state and skips the table probe; most successors of a
                                    level lead into the levels just before and after it.
                                    0 = off, 1..26 = 2^n, 0xFFFFFFFF = automatic
                                    (gx_default_opts): 2^23 entries (64 MiB) for 1- and
                                    2-word vectors in tables of at least 2^26 slots with one
                                    lane per bucket (group_lanes 1), else off.  Mid network:
                                    0.36 bucket reads per successor and 18.9 ms, against 0.82
                                    and 20.4 ms with the per-warp cache; small sizes
                                    (2^14-2^18) are far slower, many warps writing the same
                                    few lines */
  uint32_t guided_fused;         /* GX_DL_GUIDED: 1 = score the states an iteration inserts
                                    inside its expansion kernel (each CTA keeps them in shared
                                    memory and scores 128 at a time on the tensor cores), 0 =
                                    a separate scoring kernel over a pending buffer.  The
                                    search is the same either way */
} gx_explore_opts;

/* Fill *opts with the defaults described above. */
gx_status gx_default_opts(gx_explore_opts* opts);

/* Bytes of device workspace gx_explore needs for this network and options
 * (table + frontier ring + successor buffer + control block + deadlock buffer
 * + network tables).  When opts->table_bytes is 0 the table gets 1 GiB. */
gx_status gx_workspace_bytes(const gx_net* net, const gx_explore_opts* opts, uint64_t* bytes);

/* Full breadth-first exploration from the initial state (Sec. 3; the table
 * of Sec. 4 holds the visited set).  workspace: device pointer to at least
 * gx_workspace_bytes() bytes, 256-byte aligned, owned by the caller and
 * overwritten; NULL = the library allocates (cudaMallocAsync on `stream`) and
 * frees it before returning.  On GX_OK the results are kept in `net` for
 * gx_stats / gx_levels / gx_deadlocks.  GX_ERR_TABLE_FULL,
 * GX_ERR_FRONTIER_OVERFLOW, GX_ERR_SPIN_LIMIT end the search (results of the
 * levels completed so far are kept, marked incomplete).  Synchronises `stream`. */
gx_status gx_explore(gx_net* net, const gx_explore_opts* opts, void* workspace,
                     uint64_t workspace_bytes, void* stream);

/* Deadlock search (on-the-fly deadlock checking, Sec. 1 and Sec. 3).
 *   mode GX_DL_BFS_FIRST: breadth-first, stop after the level that met the
 *     first deadlock (every deadlock of that level is reported);
 *   mode GX_DL_BFS_ALL: full exploration, every deadlock reported;
 *   mode GX_DL_GUIDED: best-first order by the scoring network set with
 *     gx_guided_set_weights: each iteration expands the guided_batch open
 *     states of the best non-empty priority bin (last in, first out), then
 *     scores the states it inserted (on the tensor cores) into their bins.  Every state is pushed and eventually
 *     expanded, so the search is exhaustive: it stops at the first deadlock
 *     (reported with its path, gx_guided_trace) and reports absence only after
 *     the whole state space was explored.  Workspace: gx_guided_workspace_bytes.
 * out_states: host pointer receiving up to cap deadlock states, n_procs
 * local states each (uint32); *n_found gets the total number found (may
 * exceed cap).  Other arguments as for gx_explore. */
enum { GX_DL_BFS_FIRST = 0, GX_DL_BFS_ALL = 1, GX_DL_GUIDED = 2 };
gx_status gx_find_deadlocks(gx_net* net, const gx_explore_opts* opts, uint32_t mode,
                            void* workspace, uint64_t workspace_bytes, void* stream,
                            uint32_t* out_states, uint32_t cap, uint64_t* n_found);

/* Results of the last gx_explore / gx_find_deadlocks on `net`. */
typedef struct gx_stats_t {
  uint64_t states;          /* distinct states found (all levels) */
  uint64_t explored;        /* states whose successors were generated */
  uint64_t transitions;     /* sum over explored states of their successor count,
                               with multiplicity */
  uint64_t n_levels;        /* BFS levels found; level 0 = {initial state} */
  uint64_t deadlock_count;  /* explored states without successors */
  uint64_t deadlock_sum;    /* order-free digest of the deadlock set: sum and xor of */
  uint64_t deadlock_xor;    /* h(state) = fold_p sm64(h ^ (p << 32 | s_p)), h0 = 0 */
  int64_t first_deadlock_level; /* -1 if none */
  uint64_t table_slots;     /* slots in the hash table */
  uint32_t vector_words, slot_words, bucket_words, group_lanes, hash_rounds;
  uint32_t complete;        /* 1 = the search ended because no open state was left */
  uint32_t status;          /* gx_status of the run */
  uint32_t region_passes;   /* passes per level of the direct path (gx_explore_opts) */
  double fill;              /* states / table_slots */
  double gpu_ms;            /* device time of the search (CUDA events around it) */
  double expand_ms;         /* summed device time of the level-expansion kernels */
  uint64_t expand_launches; /* level-expansion kernel launches */
  uint64_t probes;          /* buckets read by find-or-put during the search */
  uint64_t h2d_bytes;       /* host-to-device bytes the search copied (network tables) */
  uint64_t d2h_bytes;       /* device-to-host bytes it copied (progress, deadlock states) */
  uint64_t partitioned_levels; /* levels expanded by the partitioned path */
  uint64_t violation_count; /* explored states violating the watched property (opts.watch) */
  uint64_t violation_sum;   /* order-free digest of the violation set, as for deadlocks */
  uint64_t violation_xor;
  int64_t first_violation_level; /* -1 if none */
  uint64_t kernel_launches; /* kernels the search launched (initialisation, expansion,
                               level-advance steps) */
  uint64_t device_levels;   /* levels expanded by the device-driven loop */
  uint64_t global_cache_entries; /* entries of the GPU-wide cache used (0 = not used) */
} gx_stats_t;

/* Copy the statistics of the last search on `net` into *out (host memory).
 * GX_ERR_STATE if no search has run on it yet.  Host-only. */
gx_status gx_stats(const gx_net* net, gx_stats_t* out);

/* Level sizes of the last search: out[k] = number of states at BFS depth k.
 * Writes min(cap, n_levels) entries; *n_levels gets the total. */
gx_status gx_levels(const gx_net* net, uint64_t* out, uint32_t cap, uint32_t* n_levels);

/* Per expanded level of the last gx_explore / BFS search (level k expands the
 * states of level k into level k + 1): device time in ms (CUDA events around
 * the level's kernels), buckets read by find-or-put, and successors generated.
 * Any output may be NULL; writes min(cap, n) entries, *n gets the count. */
gx_status gx_level_profile(const gx_net* net, double* ms, uint64_t* probes, uint64_t* transitions,
                           uint32_t cap, uint32_t* n);

/* Deadlock states kept by the last search (at most opts.deadlock_cap), n_procs
 * local states each, in no particular order.  *n gets the number written. */
gx_status gx_deadlocks(const gx_net* net, uint32_t* out, uint32_t cap, uint32_t* n);

/* Violating states kept by the last search with opts.watch set (at most
 * opts.violation_cap), n_procs local states each, in no particular order.
 * *n gets the number written. */
gx_status gx_violations(const gx_net* net, uint32_t* out, uint32_t cap, uint32_t* n);

/* Digest of every state in the hash table after a search: count, sum and xor
 * of h(state) (same h as the deadlock digest).  workspace/stream must be the
 * ones of the last search (the table is read in place). */
gx_status gx_set_digest(gx_net* net, void* workspace, uint64_t workspace_bytes, void* stream,
                        uint64_t* count, uint64_t* sum, uint64_t* xr);

/* ------------------------------------------------------------------------------------------
 * Learned guidance for deadlock search (no counterpart in the paper; the
 * exhaustive search it reorders is the one of Sec. 3).
 *
 * Scoring network: x = bf16(hist * (1 / n)) where hist[i] = number of
 * processes whose local state is i and n = sum of hist (the one-hot local
 * states averaged over processes, so the input has the same scale at every
 * network size; networks used with it have at most 16 local states per
 * process; an all-zero row gives x = 0), then
 * h1 = bf16(relu(W1 x + b1)) (128 x 16), h2 = relu(W2 h1 + b2) (128 x 128),
 * y = w3 . h2 + b3, trained to predict distance-to-deadlock / max_dist.  The
 * parameters are one FP32 vector W1 | b1 | W2 | b2 | w3 | b3 (GX_MLP_PARAMS
 * floats, device memory); every kernel uses the weights rounded to BF16
 * (round to nearest even), so each layer is a BF16 x BF16 product (x and h1
 * are rounded from FP32) accumulated in FP32.  Scoring (gx_mlp_forward and
 * the guided search) runs on the tensor cores, 128 states per tile.
 * ---------------------------------------------------------------------------------------- */
#define GX_MLP_IN 16
#define GX_MLP_HIDDEN 128
#define GX_MLP_PARAMS (GX_MLP_HIDDEN * GX_MLP_IN + GX_MLP_HIDDEN + GX_MLP_HIDDEN * GX_MLP_HIDDEN + \
                       GX_MLP_HIDDEN + GX_MLP_HIDDEN + 1)
/* CTAs of the gradient kernel at most; each writes its own partial gradient,
 * which a second kernel sums in a fixed order (gradients are deterministic). */
#define GX_MLP_GRAD_CTAS 256
/* Device bytes of the optimiser state gx_mlp_train needs for a batch size:
 * Adam moments, the gradient, the partial gradients and the batch indices. */
#define GX_MLP_STATE_BYTES(batch) \
  (4ull * ((3ull + GX_MLP_GRAD_CTAS) * GX_MLP_PARAMS + GX_MLP_GRAD_CTAS + 2ull) + 8ull * (batch))

/* Training examples from the last gx_explore on `net` (same workspace): every
 * state found gets its distance to the nearest deadlock (backward
 * breadth-first search over the explored graph, run as level-by-level
 * relaxation on the device: a state is at distance r when one of its
 * successors is at r - 1).  Writes up to cap examples: hist_out (device,
 * 16 uint8 per example) and label_out (device, float: min(distance, max_dist)
 * / max_dist, 1.0 when no deadlock is reachable).  dist_scratch: device, one
 * uint32 per table slot (gx_stats table_slots).  *n_out = states found (may
 * exceed cap).  The examples come sorted by content (the 16 histogram bytes,
 * then the label's bits, as unsigned words), so with cap >= *n_out the output
 * is the same on every run; the sort takes 20 bytes of temporary device
 * memory per example, the count rounded up to a power of two
 * (cudaMallocAsync on `stream`).  GX_ERR_INVALID if a process has more than 16
 * local states. */
gx_status gx_training_set(gx_net* net, void* workspace, uint64_t workspace_bytes, void* stream,
                          uint32_t* dist_scratch, uint32_t max_dist, uint8_t* hist_out,
                          float* label_out, uint64_t cap, uint64_t* n_out);

/* Seeded initialisation of params (device, GX_MLP_PARAMS floats): weights
 * uniform in +-1/sqrt(fan_in) from a splitmix64 stream, biases 0. */
gx_status gx_mlp_init(float* params, uint64_t seed, void* stream);

/* Scores of n examples (hist: device, 16 uint8 each, row-major) into out
 * (device, n floats), on the tensor cores.  Synchronises `stream`.  The
 * weights are first packed into one library-owned buffer per device, so
 * concurrent calls from several host threads run one after another.
 * GX_ERR_SPIN_LIMIT if a wait for a tensor-core product timed out. */
gx_status gx_mlp_forward(const float* params, const uint8_t* hist, uint64_t n, float* out, void* stream);

/* Self-test of failure detection without a GPU fault.  Every wait of the
 * library's kernels on an mbarrier (the tensor-core products of the scorer)
 * polls at most a fixed number of times and then reports GX_ERR_SPIN_LIMIT.
 * This call runs that bounded wait on an mbarrier that nothing arrives on, for
 * spin_limit polls (1..2^22), in one warp.  It returns GX_ERR_SPIN_LIMIT when
 * the wait gave up, which is the expected outcome; the context stays usable.
 * GX_ERR_INVALID for spin_limit 0 or above 2^22.  Synchronises `stream`. */
gx_status gx_wait_selftest(uint32_t spin_limit, void* stream);

/* Gradient of the mean squared error over n examples at params (grad: device,
 * GX_MLP_PARAMS floats, overwritten; loss: device, one float), on the tensor
 * cores: per tile of 128 examples the forward pass, then the backward products
 * D2 W2, D2^T [h1 | 1] and DA1^T [x | 1] as tcgen05 MMAs (D2 and DA1, the
 * backward signals of the two layers, enter them rounded to BF16; the bias
 * gradients come from the ones columns), accumulated in TMEM.  The result does
 * not depend on scheduling (each CTA sums its tiles in order, the partial
 * gradients are summed in a fixed order); scratch for them is allocated on
 * `stream` and freed before returning.  Synchronises `stream`;
 * GX_ERR_SPIN_LIMIT if a wait for a tensor-core product timed out. */
gx_status gx_mlp_grad(const float* params, const uint8_t* hist, const float* label, uint64_t n,
                      float* grad, float* loss, void* stream);

/* `steps` Adam steps (lr, beta 0.9 / 0.999) on mini-batches of `batch`
 * examples drawn by a counter-based stream from `seed`.  state: device,
 * GX_MLP_STATE_BYTES(batch) bytes (overwritten); loss: device, one float per
 * step (the mini-batch loss).  Synchronises `stream`. */
gx_status gx_mlp_train(float* params, float* state, const uint8_t* hist, const float* label, uint64_t n,
                       uint32_t batch, uint32_t steps, float lr, uint64_t seed, float* loss, void* stream);

/* Scoring weights for GX_DL_GUIDED searches on `net`: a device pointer to
 * GX_MLP_PARAMS floats that must stay valid while such searches run. */
gx_status gx_guided_set_weights(gx_net* net, const float* params);

/* Workspace bytes for a GX_DL_GUIDED search (table, priority bins, the log of
 * expanded states with their parents).  The bins together hold one entry per
 * table slot (a full bin spills into the next one), the log one per slot. */
gx_status gx_guided_workspace_bytes(const gx_net* net, const gx_explore_opts* opts, uint64_t* bytes);

/* The path of the deadlock found by the last GX_DL_GUIDED search: up to cap
 * states (n_procs local states each, host memory), from the initial state to
 * the deadlock; *len gets the path length in states. */
gx_status gx_guided_trace(const gx_net* net, uint32_t* out, uint32_t cap, uint32_t* len);

/* ------------------------------------------------------------------------------------------
 * Batched exploration of many independent networks (no counterpart in the
 * paper, which explores one network per run; each network is explored exactly
 * as by gx_explore).  All networks advance one BFS level per iteration inside
 * one persistent kernel launch; the iterations run on the device as a CUDA
 * graph with a conditional WHILE node, so one graph launch explores the whole
 * batch.  Narrower vectors are padded to the batch's widest slot.
 * ---------------------------------------------------------------------------------------- */
typedef struct gx_batch gx_batch;

typedef struct gx_batch_opts {
  uint32_t bucket_words;    /* 4, 8, 16 or 32; 0 = 8 */
  uint32_t group_lanes;     /* 1, 2 or 4 (see gx_batch_autotune for the built pairs); 0 = 1 */
  uint32_t hash_rounds;     /* 1..64; 0 = 8 */
  uint32_t chunk_states;    /* frontier states a warp claims at a time, a multiple of 32
                               up to 4096; 0 = 32 */
  uint64_t table_slots;     /* per-network table slots when expected_states is NULL
                               (rounded up to a power of two); 0 = 2^20 */
  const uint64_t* expected_states; /* optional host array, one entry per network: network i
                               gets a table of at least expected_states[i] / 0.75 slots */
  uint32_t levels_cap;      /* BFS levels kept per network; 0 = 4096 */
  uint32_t wide_factor;     /* an iteration with at most wide_factor x (warps of the
                               expansion grid) states, over all networks, expands one
                               warp per state (lane l takes successors l, l + 32, ...);
                               0 = 4; GX_BATCH_WIDE_OFF: never */
} gx_batch_opts;
#define GX_BATCH_WIDE_OFF 0xFFFFFFFFu

/* Make a batch from encoded networks (their encodings are copied; the
 * networks may be freed afterwards).  Host-only. */
gx_status gx_batch_create(const gx_net* const* nets, uint32_t n, gx_batch** out);
/* Free a batch and its cached graph (NULL is a no-op); the workspace belongs
 * to the caller. */
void gx_batch_free(gx_batch* batch);

/* Device workspace bytes for gx_batch_explore with these options. */
gx_status gx_batch_workspace_bytes(const gx_batch* batch, const gx_batch_opts* opts, uint64_t* bytes);

/* Explore every network of the batch (one graph launch).  workspace: device
 * pointer, 256-byte aligned, at least gx_batch_workspace_bytes bytes (required).
 * The instantiated graph is cached in the batch for the same workspace and
 * options.  Per-network results via gx_batch_stats / gx_batch_levels; the first
 * failing network's error is returned (the others' results stay valid).
 * Synchronises `stream`. */
gx_status gx_batch_explore(gx_batch* batch, const gx_batch_opts* opts, void* workspace,
                           uint64_t workspace_bytes, void* stream);

/* Results of network i in the last gx_batch_explore (gpu_ms is the whole batch). */
gx_status gx_batch_stats(const gx_batch* batch, uint32_t i, gx_stats_t* out);
/* Level sizes of network i in the last gx_batch_explore, as gx_levels does for
 * one network: min(cap, n) entries to out (host), *n_levels the total. */
gx_status gx_batch_levels(const gx_batch* batch, uint32_t i, uint64_t* out, uint32_t cap,
                          uint32_t* n_levels);

/* Autotuner: times the whole batch for every built (bucket_words, group_lanes)
 * pair -- (4,1) (8,1) (8,2) (16,1) (16,2) (32,2) (32,4), those not narrower than
 * the slots -- and chunk_states 32, 64, 128 (median of three runs each, CUDA
 * events), then writes the fastest into *opts (other fields kept) and its time
 * into *best_ms.  The workspace must fit every candidate (all need the same). */
gx_status gx_batch_autotune(gx_batch* batch, gx_batch_opts* opts, void* workspace,
                            uint64_t workspace_bytes, void* stream, double* best_ms);

/* ------------------------------------------------------------------------------------------
 * Exploration that allocates nothing.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory -- a host
 * framework that has reserved the GPU's memory for its own pool (cudaMalloc
 * then fails or escapes its accounting), or a latency-critical caller that
 * must not pay cudaFree's device-wide synchronisation.
 *
 * The breadth-first search of gx_explore (levels driven from the host, one
 * control-block read per level), but all scratch (control block, network
 * tables, frontier ring, hash table, GPU-wide cache) lives in one static
 * device array of
 * GX_NOALLOC_SCRATCH_BYTES inside the library, which every GPU that loads the
 * library holds until the process exits.  No cudaMalloc, cudaFree or other
 * allocating call is made.
 *   - Options honoured as by gx_explore: bucket_words, group_lanes,
 *     hash_rounds, table_bytes (0 means 32 MiB here), frontier_states,
 *     ctas_per_sm, max_levels, stop_at_first_deadlock, warp_cache_log2 (the
 *     cache is shared memory only), global_cache_log2 (its entries come from
 *     the array), region_passes (0 means 1 here), and the safety check
 *     (watch, watch_proc, watch_state, stop_at_first_violation).
 *   - Not used: deadlock_cap and violation_cap (deadlocks and violations are
 *     counted and digested but no state is stored), host_loop (the levels are
 *     always driven from the host), slice_log2 and successor_buffer (they only
 *     apply to the partitioned path), and the guided_* fields (BFS only).
 *   - Rejected with GX_ERR_INVALID: partition_min_states other than 0 (the
 *     partitioned path needs a successor buffer); sizes for which table +
 *     frontier + network tables + cache exceed the array (the message gives
 *     them).
 *   - Outputs: *stats_out (gpu_ms and expand_ms are 0: no events are
 *     created); levels_out receives min(levels_cap, n) level sizes and
 *     *n_levels (may be NULL) the total.  Nothing is recorded in `net`.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) and caches it; make that first call before any
 *     stream capture.
 *   - Every call shares the array and it keeps the previous call's contents;
 *     each call clears what must start at zero.  Calls whose device work
 *     overlaps (two streams, two threads) race on the array.
 * Synchronises `stream`. */
#define GX_NOALLOC_SCRATCH_BYTES (64ull << 20)
gx_status gx_explore_noalloc(const gx_net* net, const gx_explore_opts* opts, void* stream,
                             gx_stats_t* stats_out, uint64_t* levels_out, uint32_t levels_cap,
                             uint32_t* n_levels);

/* ------------------------------------------------------------------------------------------
 * The isolated hash-table experiment (Sec. 5.1, Fig. "buckvsgputable"):
 * find-or-put of n_keys keys of key_words uint32 each into a table.
 *   keys:    device pointer, n_keys * key_words uint32, row-major; bit 31 of
 *            every word must be clear (the table uses it as the occupied tag).
 *   table:   device pointer, table_words uint32 (a power-of-two multiple of
 *            bucket_words, 256-byte aligned).  Zero it first for an empty
 *            table; it is read and written in place.
 *   result:  device pointer, n_keys bytes, or NULL: 1 = this call inserted the
 *            key, 0 = the key was already present, 2 = no free slot in any round.
 *   counters: device pointer to 3 uint64 (inserted, found, failed), added to.
 * key_words: 1, 2 or 4; bucket_words, group_lanes, hash_rounds as in
 * gx_explore_opts (0 = default).  The keys are taken by a grid-stride loop on
 * 16 times the CTAs that fit at once (random reads run faster from such a grid
 * than from a resident one).  Asynchronous on `stream`. */
gx_status gx_find_or_put(const uint32_t* keys, uint64_t n_keys, uint32_t key_words,
                         uint32_t bucket_words, uint32_t group_lanes, uint32_t hash_rounds,
                         uint32_t* table, uint64_t table_words, uint8_t* result,
                         uint64_t* counters, void* stream);

/* Cuckoo hashing, the lock-free GPU table Sec. 4.1 weighs against its own
 * (Alcantara et al.'s GPU form of Pagh & Rodler's cuckoo hashing), for
 * comparison on the Sec. 5.1 key sequences.  One thread per key:
 *   1. lookup: the key is present if one of its n_hash positions holds it;
 *      pos_i(x) = (mix(x) * m_i mod 2^64) >> (64 - log2 table_slots), with
 *      mix the splitmix64 output function (Steele, Lea & Flood 2014) of the
 *      stored slot value x (1-word keys: the tagged word; 2-word keys: word 0
 *      | word 1 << 32, both tagged);
 *   2. otherwise the key is exchanged into pos_0.  A key y evicted from a slot
 *      p moves, by exchange, to pos_{(j+1) mod n_hash}(y), j the first index
 *      with pos_j(y) = p.  The chain ends when an exchange meets an empty slot
 *      or the key it carries; after max_chain exchanges the key still carried
 *      is dropped (result 2, counted as failed; the table then lacks a key).
 * A key being moved sits in no slot, so a concurrent lookup of it misses and
 * inserts it again: find-or-put can report one key as new more than once and
 * store it twice.  That is the property Sec. 4.1 finds missing for
 * state-space exploration.  While nothing failed, the keys stored still form
 * exactly the input's set, and one key per call gives the sequential
 * algorithm exactly.
 *   keys:     device, n_keys * key_words uint32, bit 31 of every word clear.
 *   key_words: 1 (32-bit slots) or 2 (64-bit slots).
 *   muls:     host, n_hash odd uint64 multipliers m_i, copied; NULL takes the
 *             first n_hash hash-constant sets of gx_find_or_put.
 *   table:    device, table_slots * key_words uint32, 256-byte aligned;
 *             table_slots a power of two >= 2; zeroed by the caller for an
 *             empty table; a stored word is the key word | 2^31.
 *   result:   device, n_keys bytes, or NULL: 1 = inserted, 0 = found (by the
 *             lookup, or by the first exchange meeting the key), 2 = the chain
 *             dropped a key.
 *   counters: device, 4 uint64 (inserted, found, failed, exchanges), added to.
 * n_hash 2..8 (0 = 4); max_chain 1..4096 (0 = 128).  GX_ERR_INVALID for other
 * values, an even multiplier, NULL or misaligned pointers.  One thread per key,
 * on the same grid shape as gx_find_or_put (16 times the CTAs that fit at
 * once).  Asynchronous on `stream`. */
gx_status gx_cuckoo_find_or_put(const uint32_t* keys, uint64_t n_keys, uint32_t key_words,
                                uint32_t n_hash, uint32_t max_chain, const uint64_t* muls,
                                uint32_t* table, uint64_t table_slots, uint8_t* result,
                                uint64_t* counters, void* stream);

/* Random-access probes used as the roofline for the table (no counterpart in
 * the paper): over the largest power-of-two number of `bytes`-sized units that
 * fits a device buffer of `words` uint32, `n` accesses at pseudo-random
 * unit-aligned positions, each reading `bytes` (16, 32, 64 or 128) contiguous
 * bytes (kind 0) or doing one 32/64/128-bit compare-and-swap (kind 1, `bytes`
 * = 4, 8 or 16).  sink: device pointer to one uint64 that
 * receives a checksum so the reads cannot be optimised away.  Asynchronous. */
gx_status gx_probe_random(uint32_t kind, uint32_t* buffer, uint64_t words, uint64_t n,
                          uint32_t bytes, uint64_t seed, uint64_t* sink, void* stream);

/* Random gathers with a chosen launch shape and locality, for measuring the
 * ceiling the table's random accesses are held against (no counterpart in the
 * paper).  Over the largest power-of-two number of unit_bytes-sized units (32,
 * 64 or 128: one sector, or the bucket sizes of 16 and 32 words) that fits
 * `words` uint32 of `buffer`, `n` accesses at counter-based pseudo-random unit
 * positions (mix64(seed + i), as gx_probe_random):
 *   load_bytes:  4 = read one word of the unit (the DRAM still moves the whole
 *                sector; one register per access in flight), or unit_bytes =
 *                read the whole unit with 256-bit loads;
 *   in_flight:   accesses each thread issues before it uses any: 1, 2, 4, 8,
 *                16, or 32 (4-byte loads only); at most 4 with 128-byte loads;
 *   ctas_per_sm: 256-thread CTAs per SM: 1..8, lowered to what the kernel's
 *                registers allow (a grid resident at once); 9..32 as asked (a
 *                grid of more than one wave, whose CTAs finish and start during
 *                the launch); *ctas_used (host, may be NULL) gets the value
 *                launched (the grid is SMs x ctas_used);
 *   group_log2:  0 = every access independent; g >= log2(unit_bytes) = the
 *                accesses a warp issues together (32 x in_flight) fall in one
 *                randomly chosen aligned block of 2^g bytes (page locality).
 * buffer: device, 256-byte aligned (an offset into a larger allocation
 * measures one region of it).  sink: device, one uint64 receiving a checksum.
 * GX_ERR_INVALID for other values.  Asynchronous on `stream`. */
gx_status gx_probe_gather(uint32_t* buffer, uint64_t words, uint64_t n, uint32_t unit_bytes,
                          uint32_t load_bytes, uint32_t in_flight, uint32_t ctas_per_sm, uint32_t group_log2,
                          uint64_t seed, uint64_t* sink, void* stream, uint32_t* ctas_used);

#ifdef __cplusplus
}
#endif
#endif /* GX_H */
