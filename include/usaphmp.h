/*
 * usaphmp.h -- C ABI of the GB300 library for the Uncapacitated Single
 * Allocation p-Hub Median Problem (USApHMP): batched fitness evaluation of a
 * population of chromosomes and the device-side step of the island GA of
 * Benaini, Berrajaa, Boukachour and Oudani, "Solving the Uncapacitated Single
 * Allocation p-Hub Median Problem on GPU" (arXiv 1704.06258).
 *
 * Problem (§3, eq. 1-5): n nodes, flows W[i][j] >= 0, unit costs
 * C[i][k] >= 0; open exactly p hubs and allocate every node to one open hub
 * (each hub to itself) to minimise
 *     sum_i sum_j W[i][j] * (chi*C[i][h(i)] + alpha*C[h(i)][h(j)] + delta*C[h(j)][j]),
 * the hub-to-hub leg taken on the direct arc (a shortest hub path whenever C
 * satisfies the triangle inequality, e.g. Euclidean C).
 *
 * Chromosome encoding (§4.1): the p open hubs (node ids 0..n-1) and the
 * allocation S, S[i] = the hub serving node i, S[k] = k for every hub k.
 *
 * Conventions.
 *  - All matrices are row-major, node ids are 0-based.
 *  - Functions return 0 (USAPHMP_OK) or a negative USAPHMP_E* code; the
 *    message of the last failure of the calling thread is returned by
 *    usaphmp_last_error().
 *  - Host-pointer functions copy their inputs before returning and never keep
 *    caller pointers.  *_dev functions take device pointers and a
 *    cudaStream_t (passed as void*; NULL = the legacy default stream) and are
 *    ordered on that stream; they return after enqueueing unless stated.
 *  - A handle is not thread-safe: calls on one handle must not overlap.
 *  - The library needs an sm_103 GPU; there is no CPU fallback.
 */
#ifndef USAPHMP_H
#define USAPHMP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  USAPHMP_OK = 0,
  USAPHMP_EINVAL = -1,        /* bad argument: size, null pointer, NaN/Inf/negative W or C */
  USAPHMP_EINVAL_CHROM = -2,  /* a chromosome violates eq. (2), (3) or (5) */
  USAPHMP_ENOMEM = -3,        /* device allocation failed */
  USAPHMP_ECUDA = -4,         /* a CUDA call failed (message names it) */
  USAPHMP_ETIMEOUT = -5,      /* a device-side wait gave up (kernel returned early) */
  USAPHMP_EBUSY = -6,         /* resource limit reached (admission refused) */
  USAPHMP_EIO = -7,           /* a file could not be written */
  USAPHMP_ECANCELED = -8      /* the request was cancelled (usaphmp_server_cancel) */
};

/* Transfer leg of objective (1) between the hubs h(i) and h(j) (eq. 4 lets
 * flow take any path between hubs).  DIRECT: the arc C[h(i)][h(j)], a
 * shortest path whenever C satisfies the triangle inequality.  HUB_PATHS:
 * the cheapest path over arcs between the chromosome's open hubs
 * (Floyd-Warshall on its p x p hub costs, §3 defines Y^i_kl as flow between
 * hubs k and l); a pair served by one hub has no transfer leg.  For C with a
 * zero diagonal and the triangle inequality both give the same cost up to
 * rounding. */
enum {
  USAPHMP_ROUTE_DIRECT = 0,
  USAPHMP_ROUTE_HUB_PATHS = 1
};

/* Scale of the objective values returned to the caller (§4.3: the CAB
 * benchmarks report the cost per unit of flow, the AP/Urand ones the cost
 * times 10^-3, PlanetLab the raw cost).  It multiplies the fitness written by
 * usaphmp_eval / _eval_dev / _eval_slots_dev (in fp32), the costs of
 * usaphmp_rescore_fp64_dev (in fp64) and both costs of a result; the GA
 * selects on the raw cost, so the search is the same for every scale.
 * PER_FLOW divides by sum_ij W[i][j] (computed in fp64 at creation; refused
 * when it is 0). */
enum {
  USAPHMP_SCALE_RAW = 0,
  USAPHMP_SCALE_MILLI = 1,
  USAPHMP_SCALE_PER_FLOW = 2
};

/* Evaluators of the transfer term. */
enum {
  USAPHMP_PATH_PLAIN_FP32 = 0,  /* fp32 CUDA cores, shared-memory gather of C[h(i)][h(j)] */
  USAPHMP_PATH_SPLIT_BF16 = 1,  /* tcgen05 GEMM W*A with W = bf16 hi + lo, fp32 accumulation */
  USAPHMP_PATH_FP64_REF = 2     /* reference: the pair form of eq. 1 in fp64 for every chromosome
                                   (the rescoring kernels), rounded to the fp32 fitness; slow,
                                   for checks; not offered by the server */
};

typedef struct usaphmp_s* usaphmp_t;

/* GA parameters (§5 names R islands of size n, N1 inner and N2 outer
 * iterations without values; these are the library's choices). */
typedef struct {
  int32_t islands;      /* R >= 1 (default 64) */
  int32_t island_size;  /* P, even, >= 2 (default 64); population B = R*P */
  int32_t n1;           /* generations between island merges (default 10);
                           0: never merge (a caller sharding islands over GPUs
                           merges them with usaphmp_ga_islands / _ga_merge) */
  int32_t path;         /* USAPHMP_PATH_* (default SPLIT_BF16) */
  int32_t elitist;      /* 0 (default): ancestor = best child unconditionally */
  int32_t use_graph;    /* 1 (default): replay generations from a CUDA graph */
  int32_t routing;      /* USAPHMP_ROUTE_* (default DIRECT); applies to every
                           evaluation, generation and fp64 rescoring of the
                           handle (the server and the allocation-free entry
                           point use DIRECT) */
  int32_t scale;        /* USAPHMP_SCALE_* (default RAW) */
  int32_t local_search; /* >= 0 (default 0): sweeps of the allocation local
                           search (usaphmp_local_search_dev) applied to the
                           returned solution; the GA itself evaluates nearest
                           allocations */
  int32_t island_offset; /* >= 0 (default 0): global index of this handle's
                            first island.  Random streams are addressed by the
                            global chromosome index (island_offset + r) * P + j,
                            so shards of one island population over several
                            GPUs draw what one GPU holding all islands draws */
} usaphmp_params;

typedef struct {
  int32_t* hubs;      /* out [p], caller-allocated: best hubs, ascending */
  int32_t* S;         /* out [n], caller-allocated: their nearest allocation */
  double cost_fp64;   /* objective of (hubs, S) rescored in fp64 */
  float cost_fp32;    /* the fast path's fitness of the same solution */
  int64_t evals;      /* chromosome evaluations performed */
  double ms;          /* wall time of the call */
} usaphmp_result;

/* Creates an instance: copies W and C (host, n*n floats each) to the device,
 * checks them (finite, >= 0), computes O, D, whether C is symmetric and the
 * bf16 split of the tensor-core operand: W, or for symmetric C the folded
 * U = W + W^T above the diagonal (W_ii on it), which halves the transfer
 * GEMM.  2 <= n <= 16384, 1 <= p <= min(n, 255).  Defines: §3. */
int usaphmp_create(int32_t n, int32_t p, const float* W, const float* C, double chi,
                   double alpha, double delta, usaphmp_t* out);

/* Same with device W and C (n*n floats, row-major), read on `stream`; the
 * call synchronises `stream` before returning. */
int usaphmp_create_dev(int32_t n, int32_t p, const float* W, const float* C, double chi,
                       double alpha, double delta, void* stream, usaphmp_t* out);

int usaphmp_set_params(usaphmp_t h, const usaphmp_params* prm);
int usaphmp_get_params(usaphmp_t h, usaphmp_params* prm);

/* What the instance holds (read-only). */
typedef struct {
  int32_t n, p;
  int32_t ldw;           /* row stride of the device matrices (n rounded up to 8) */
  int32_t ns;            /* row stride of the slot codes (n rounded up to 64) */
  int32_t c_symmetric;   /* 1 when C equals its transpose bit for bit */
  int32_t tc_folded;     /* 1 when the tensor-core operand is the folded U (only the
                            K blocks right of each row block's diagonal are multiplied) */
} usaphmp_info;
int usaphmp_get_info(usaphmp_t h, usaphmp_info* info);

/* Fitness (objective 1 times the handle's output scale, raw by default) of B
 * chromosomes given on the host in the encoding of §4.1: hubs [B][p] node ids
 * (any order), S [B][n] node ids; fitness [B] out.  Computed on the GPU by the
 * configured path (fp32 arithmetic): the inputs are copied in chunks, each
 * chunk checked and put in canonical form as it lands, and the call returns
 * once the fitness is on the host (the caller's buffers are not retained).
 * Returns USAPHMP_EINVAL_CHROM naming the first invalid chromosome (eq. 2, 3,
 * 5: distinct hubs, S[i] an open hub, every hub serving itself). */
int usaphmp_eval(usaphmp_t h, int32_t B, const int32_t* hubs, const int32_t* S, double* fitness);

/* Same with device arrays; fitness is fp32 [B].  Validation needs the device
 * status word, so this call synchronises `stream` before returning. */
int usaphmp_eval_dev(usaphmp_t h, int32_t B, const int32_t* hubs, const int32_t* S,
                     float* fitness, void* stream);

/* Runs the GA (§5): middle-node initial solution (§4.1), `generations`
 * generations of offspring + nearest allocation + evaluation + selection on
 * the device, then fp64 rescoring of the best-ever solution. */
int usaphmp_solve(usaphmp_t h, int32_t generations, uint64_t seed, usaphmp_result* best);

void usaphmp_destroy(usaphmp_t h);
const char* usaphmp_last_error(void);

/* ---------------------------------------------------------------------------
 * Step-level entry points on the library's internal layouts (device pointers,
 * ordered on `stream`, no synchronisation, no validation).
 *   mask  u32 [B][nw]  bit i%32 of word i/32 set <=> node i is a hub
 *   hubs  i32 [B][p]   open hubs in ascending node order
 *   slot  u8  [B][ns]  rank in `hubs` of the hub serving node i (ns >= n;
 *                      bytes n..ns-1 are padding, written as 0xFF)
 * ------------------------------------------------------------------------- */
int usaphmp_layout(usaphmp_t h, int32_t* ns, int32_t* nw);

/* Middle-node initial solution (§4.1): the p nodes with the smallest
 * sum_j C[i][j] (lower id on ties).  mask [nw], hubs [p] out. */
int usaphmp_initial_dev(usaphmp_t h, uint32_t* mask, int32_t* hubs, void* stream);

/* Offspring of generation g for R islands of P members (§4.1, §4.2, §5):
 * exchange, crossover, mutation, correction, driven by Philox4x32-10 draw
 * streams of `seed`.  anc [R][nw] in; mask [R*P][nw] and hubs [R*P][p] out. */
int usaphmp_children_dev(usaphmp_t h, int32_t R, int32_t P, const uint32_t* anc, uint64_t seed,
                         int32_t g, uint32_t* mask, int32_t* hubs, void* stream);

/* Nearest-hub allocation (§4.1, §5): slot [B][ns] out from ascending hubs
 * (slot 4-byte aligned, else USAPHMP_EINVAL). */
int usaphmp_allocate_dev(usaphmp_t h, int32_t B, const int32_t* hubs, uint8_t* slot, void* stream);

/* Fitness (fp32 [B] out) of chromosomes in canonical form (ascending hubs,
 * slot codes [B][ns], 4-byte aligned, padding 0xFF) by the configured path.
 * Uses the handle's scratch buffers. */
int usaphmp_eval_slots_dev(usaphmp_t h, int32_t B, const int32_t* hubs, const uint8_t* slot,
                           float* fitness, void* stream);

/* Selection of generation g (§5) for R islands of P members: ancestors
 * anc [R][nw] / anc_fit [R], best-ever best [nw] / best_fit [1] updated in
 * place from the children mask [R*P][nw] and their fitness [R*P]. */
int usaphmp_select_dev(usaphmp_t h, int32_t R, int32_t P, int32_t g, const uint32_t* mask,
                       const float* fitness, uint32_t* anc, float* anc_fit, uint32_t* best,
                       float* best_fit, void* stream);

/* Island exchange for a population sharded over GPUs (§5 outer loop; the
 * caller moves the data between processes).  usaphmp_ga_islands copies the
 * current ancestors (host, [R][nw] words, bit i%32 of word i/32 = node i)
 * and their fitness (host, [R] raw fp32 costs); either output may be NULL.
 * usaphmp_ga_merge sets every island's ancestor to `mask` (host, nw words,
 * exactly p bits among the first n) with fitness `fit`: the merge the GA
 * does itself every n1 generations when all islands are on one GPU (run
 * with n1 = 0 and call this after every n1 generations).  Both need
 * usaphmp_ga_begin first and synchronise `stream`. */
int usaphmp_ga_islands(usaphmp_t h, uint32_t* masks, float* fit, void* stream);

/* The population of the last generation run (§5): the children's hub masks
 * (host, [R*P][nw] words, chromosome q = r*P + j of island r) and their raw
 * fp32 fitness (host, [R*P]) as the selection saw them; before the first
 * generation their contents are unspecified.  Either output may be NULL.
 * Needs usaphmp_ga_begin first; synchronises `stream`. */
int usaphmp_ga_population(usaphmp_t h, uint32_t* masks, float* fit, void* stream);
int usaphmp_ga_merge(usaphmp_t h, const uint32_t* mask, float fit, void* stream);

/* Checkpoint / resume of the GA between generations.  The state is small:
 * the island ancestors and their fitness, the best-ever solution, the
 * generation counter and the seed (the random streams are counter-based, so
 * a resumed run draws exactly what an uninterrupted one draws).  A state
 * saved by usaphmp_ga_save (after usaphmp_ga_begin) and loaded by
 * usaphmp_ga_load into a handle of the same instance size and GA parameters
 * continues the run bit for bit.  bytes = usaphmp_ga_state_bytes for the
 * handle's current parameters; a buffer of another size, with another
 * layout version or saved with other n, p, islands, island_size, n1, elitist
 * or island_offset gives USAPHMP_EINVAL (nothing changed).  Both calls
 * synchronise `stream`. */
int usaphmp_ga_state_bytes(usaphmp_t h, int64_t* bytes);
int usaphmp_ga_save(usaphmp_t h, void* buf, int64_t bytes, void* stream);
int usaphmp_ga_load(usaphmp_t h, const void* buf, int64_t bytes, void* stream);

/* Allocation local search for fixed hubs, in fp64 (§4.1 allocates every
 * spoke to its nearest hub, which is not always the cheapest allocation for
 * those hubs).  A sweep visits the spokes in ascending node order and moves
 * spoke i to the open hub whose choice lowers objective (1) the most (the
 * lowest node id among equal changes), when the change is negative, before
 * visiting the next spoke; sweeps repeat until one moves nothing or
 * max_sweeps (>= 1) have run.  Hubs keep serving themselves.  Uses the
 * handle's routing.
 *   hubs  i32 [B][p] ascending node ids (device)
 *   slot  u8  [B][ns] (device, in/out): rank in hubs of each node's hub,
 *         a valid single allocation on entry (every hub in its own slot)
 *   moves, sweeps  i32 [B] out (device, may be NULL): moves made, sweeps run
 * Scratch: B * (2*n*p + p*(p|1)) doubles, kept by the handle and grown when
 * a call needs more; the first call also makes W transposed and the fp64
 * flow sums (n*n floats + 2n doubles).  Synchronises `stream` before
 * returning. */
int usaphmp_local_search_dev(usaphmp_t h, int32_t B, const int32_t* hubs, uint8_t* slot, int32_t max_sweeps,
                             int32_t* moves, int32_t* sweeps, void* stream);

/* FP64 objective of B canonical chromosomes (§3, eq. 1 in its pair form:
 * sum_i sum_j W[i][j] (chi C[i][h(i)] + alpha T[h(i)][h(j)] + delta C[h(j)][j]),
 * T the transfer leg of the handle's routing), every product and sum in fp64
 * from the fp32 instance and the fp64 factors given at creation, times the
 * handle's output scale.
 *   hubs i32 [B][p] ascending node ids, slot u8 [B][ns] (device); cost fp64 [B]
 *   out (device).
 * Scratch (B * min(n, 128) doubles, and B*p*p more with hub-path routing) is
 * allocated for the call and freed before it returns; synchronises `stream`. */
int usaphmp_rescore_fp64_dev(usaphmp_t h, int32_t B, const int32_t* hubs, const uint8_t* slot,
                             double* cost, void* stream);

/* GA run control (what usaphmp_solve does, split for timing):
 * begin = initial solution + state; run = `generations` generations enqueued
 * on `stream` without host synchronisation; result = rescoring + copy-out. */
int usaphmp_ga_begin(usaphmp_t h, uint64_t seed, void* stream);
int usaphmp_ga_run(usaphmp_t h, int32_t generations, void* stream);
int usaphmp_ga_result(usaphmp_t h, usaphmp_result* best, void* stream);

/* usaphmp_ga_run without graph replay and with CUDA events recorded on
 * `stream` between the stages of every generation.  Synchronises `stream`
 * after each generation and adds the device time (ms) of each stage to
 * stage_ms[0..5]: 0 offspring (§4.1-4.2), 1 nearest allocation + access
 * terms, 2 transfer term (the configured evaluator), 3 fitness reduction
 * fused with selection (§5), 4 unused (0), 5 the whole generation. */
int usaphmp_ga_run_profiled(usaphmp_t h, int32_t generations, void* stream, double* stage_ms);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of GA solve requests of differing n and p on
 * one GPU.  Requests queue in FIFO order and are admitted while at most
 * `max_active` (<= 64) are admitted or running and the device bytes of those
 * (usaphmp_server_footprint) stay within `hbm_budget_bytes`; a request that
 * alone exceeds the budget finishes with USAPHMP_EBUSY.  Each
 * usaphmp_server_step admits what fits, then enqueues up to 8 generations
 * (§5) of every running request -- as many as every one of them still needs,
 * at most 8 -- with one launch per kernel and generation over all of them,
 * replayed from a CUDA graph that is captured again only when the running
 * set changes.
 * A request's result does not depend on which other requests ran beside it.
 * The step does no device-memory management and waits for no request: a
 * worker thread of the server makes each admitted request's instance
 * (stream-ordered allocations from the server's memory pool, which keeps up
 * to the budget for reuse; the set-up and the initial solution run on the
 * request's own stream) and finishes each request whose last generation has
 * been enqueued (fp64 rescoring, copy-out, release), so the step returns
 * after enqueueing, waiting only when the device is two steps behind.  The
 * server's calls must come from one thread (the worker is internal).
 * ------------------------------------------------------------------------- */
typedef struct usaphmp_server_s* usaphmp_server_t;

int usaphmp_server_create(int64_t hbm_budget_bytes, int32_t max_active, int32_t path, usaphmp_server_t* out);

/* Queues a request (W, C host n*n, copied); *ticket identifies it. */
int usaphmp_server_submit(usaphmp_server_t s, int32_t n, int32_t p, const float* W, const float* C, double chi,
                          double alpha, double delta, int32_t islands, int32_t island_size, int32_t generations,
                          uint64_t seed, int64_t* ticket);

/* One tick (see above); n_active = requests admitted (being made) or
 * running, n_pending = requests queued for admission plus requests being
 * finished; either may be NULL. */
int usaphmp_server_step(usaphmp_server_t s, int32_t* n_active, int32_t* n_pending);

/* Counters since the server was made: ticks and their host wall time (total
 * and largest, ms), requests admitted into the running set, their wait from
 * submission to joining it (total and largest, ms), the worker's time making
 * their instances (total, ms), and the ticks that captured their generation
 * graph anew. */
typedef struct {
  int64_t ticks;
  double tick_ms_total, tick_ms_max;
  int64_t admitted;
  double admit_wait_ms_total, admit_wait_ms_max;
  double admit_ms_total;
  int64_t graph_builds;   /* ticks that captured their generations anew (the others replayed) */
} usaphmp_server_counters;
int usaphmp_server_stats(usaphmp_server_t s, usaphmp_server_counters* out);

/* 1: finished, *out filled (hubs/S into caller buffers of p and n entries;
 * ms = wall time from submission to the result being ready) and the ticket
 * forgotten; 0: not finished; < 0: the request failed (message in
 * usaphmp_last_error). */
int usaphmp_server_poll(usaphmp_server_t s, int64_t ticket, usaphmp_result* out);

/* Cancels a request between steps: a queued one leaves the queue, a running
 * or admitted one stops (its slot is free at once; its device memory returns
 * to the pool once the generations already enqueued for it have run).  Its
 * poll then returns USAPHMP_ECANCELED.  USAPHMP_EINVAL for a ticket that is
 * not queued, admitted or running (unknown, finished or already cancelled). */
int usaphmp_server_cancel(usaphmp_server_t s, int64_t ticket);

/* Device bytes a request of this shape holds while it runs. */
int usaphmp_server_footprint(int32_t n, int32_t p, int32_t islands, int32_t island_size, int64_t* bytes);

void usaphmp_server_destroy(usaphmp_server_t s);

/* ---------------------------------------------------------------------------
 * Tile shapes of the tensor-core evaluator and their autotuner.  The paper
 * has no counterpart (its kernel is one thread per chromosome).
 *
 * The split-bf16 evaluator (USAPHMP_PATH_SPLIT_BF16) multiplies W by the
 * one-hot allocation matrices of the population in tiles of 128 rows x
 * ntile columns; a tile holds floor(ntile / p) whole chromosomes.  Shape:
 *   ntile   64, 128 or 256 (>= p)
 *   stages  2..4 shared-memory pipeline stages (ntile 256: at most 3 with
 *           pair 0)
 *   raster  0: the persistent CTAs walk the column tiles of one row block of
 *           W first; 1: the row blocks of one column tile first.
 *   pair    0: one CTA per MMA (M = 128); 1: clusters of two CTAs on
 *           neighbouring SMs run each MMA over two row blocks (M = 256,
 *           tcgen05 cta_group::2), each CTA staging its own row block of W
 *           and half of the one-hot columns.
 * The shape changes speed only: fitness values are bit-identical for every
 * shape.  Default {256, 3, 0}.  A handle's shape applies to its own
 * evaluations and generations; the server uses the default. */
typedef struct {
  int32_t ntile;
  int32_t stages;
  int32_t raster;
  int32_t pair;
} usaphmp_tile;

/* USAPHMP_EINVAL (nothing changed) for a shape outside the list above or
 * with ntile < p.  Drops the handle's captured generation graph. */
int usaphmp_set_tile(usaphmp_t h, const usaphmp_tile* tile);
int usaphmp_get_tile(usaphmp_t h, usaphmp_tile* tile);

/* Autotuner: times every valid shape on the handle's current population
 * size (islands * island_size chromosomes of the handle's instance) and
 * keeps the fastest as the handle's shape (ties keep the earlier candidate;
 * the default is tried first).  Each candidate runs 1 untimed and `reps`
 * timed launches (1 <= reps <= 1000) of the transfer-term kernel, measured
 * with CUDA events on the handle's stream.  The population is one GA
 * generation grown from the initial solution with a fixed seed, so the call
 * resets the GA state: call usaphmp_ga_begin (or usaphmp_solve) afterwards.
 * With cache_path non-NULL the bucket (device name, ceil(n/128), p, the
 * population size rounded up to a power of two) is first looked up in that
 * JSON file (format: usaphmp_tile_cache_store) and, when present and valid
 * for p, applied without timing (*from_cache = 1); otherwise the timed
 * choice is stored there.  Outputs may be NULL: the chosen shape, its mean
 * launch time and the default shape's (both 0 when taken from the cache).
 * On the plain path the call only returns the current shape. */
int usaphmp_autotune(usaphmp_t h, int32_t reps, const char* cache_path, usaphmp_tile* chosen,
                     double* chosen_ms, double* default_ms, int32_t* from_cache);

/* The autotuner's JSON cache, host only (no GPU needed).  usaphmp_autotune
 * keys it by the device name, followed by " (folded operand)" for instances
 * whose C is symmetric.  A file holds
 *   {"format": "usaphmp-tile-cache-1", "entries": [{"device": "...",
 *    "n_blocks": ceil(n/128), "p": p, "B_pow2": B rounded up to a power of
 *    two, "ntile": ..., "stages": ..., "raster": ..., "ms": ...}, ...]}.
 * lookup: 1 and *out (and *ms if non-NULL) filled when the bucket of
 * (device, n, p, B) is present, 0 when it is not or the file does not exist,
 * USAPHMP_EINVAL when the file is not such a JSON document.
 * store: inserts or replaces the bucket's entry, rewriting the file through
 * a temporary file and a rename (USAPHMP_EIO when that fails). */
int usaphmp_tile_cache_lookup(const char* path, const char* device, int32_t n, int32_t p, int32_t B,
                              usaphmp_tile* out, double* ms);
int usaphmp_tile_cache_store(const char* path, const char* device, int32_t n, int32_t p, int32_t B,
                             const usaphmp_tile* tile, double ms);

/* ---------------------------------------------------------------------------
 * Testing hooks (failure detection without a GPU fault).
 *
 * usaphmp_debug_fail_allocations: the next `after` device allocations of the
 * library succeed and the one after fails (the call reports USAPHMP_ENOMEM);
 * after < 0 turns the injection off.  Process-wide.
 *
 * usaphmp_selftest_wait_timeout: runs one small kernel whose threads wait,
 * with the bounded waits of the tensor-core evaluator and a limit of
 * limit_ns (1e3 .. 1e10), on a barrier that nothing completes.  Returns
 * USAPHMP_ETIMEOUT when the waits gave up as they must (status holds the
 * device status word, elapsed_ns the time the waits took); USAPHMP_ECUDA
 * otherwise.  The CUDA context stays usable. */
int usaphmp_debug_fail_allocations(int32_t after);
int usaphmp_selftest_wait_timeout(int64_t limit_ns, uint32_t* status, int64_t* elapsed_ns);

/* ---------------------------------------------------------------------------
 * Allocation-free entry point.  The paper has no counterpart: this exists for
 * callers that cannot call cudaMalloc -- code that must stay inside a device
 * memory budget or pool owned by a host application, or a latency-critical
 * loop where cudaMalloc's implicit device synchronisation is not acceptable.
 *
 * The fp64 pair form of eq. 1, as usaphmp_rescore_fp64_dev computes it for a
 * handle with the default routing and scale -- the transfer leg on the direct
 * hub arc C[h(i)][h(j)] and the raw, unscaled cost -- but without a handle:
 * every input and the output are caller device buffers, and the function
 * neither allocates nor frees anything.  Its per-block partial sums go to a
 * fixed scratch array compiled into the library: 131072 doubles (1 MiB),
 * present on every GPU that loads the library until the process exits.
 *   W, C   fp32 [n][n] row-major (dense, no padding; C need not be symmetric)
 *   hubs   i32  [B][p] ascending node ids; slot u8 [B][n] (rank in hubs of the
 *          hub serving node i); cost fp64 [B] out.
 * Sizes: 2 <= n <= 16384, 1 <= p <= min(n, 255), and B * min(n, 128) must not
 * exceed 131072 (else USAPHMP_EINVAL, nothing launched).  Enqueued on
 * `stream`, no synchronisation.
 * Set-up: the scratch array's device address is looked up once per CUDA
 * context of a device (the first call on a device, and the first call after
 * that device's context was reset), with the device current; make that first
 * call before any stream capture.  All calls share the one scratch array
 * (every call rewrites the entries it reads, nothing needs to start at zero),
 * so calls whose work overlaps on the GPU -- on different streams or from
 * different threads -- race and return wrong costs: order them on one stream
 * or synchronise between them. */
int usaphmp_rescore_fp64_noalloc(int32_t n, int32_t p, int32_t B, const float* W, const float* C,
                                 double chi, double alpha, double delta, const int32_t* hubs,
                                 const uint8_t* slot, double* cost, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* USAPHMP_H */
