/*
 * agg.h - C ABI of the GB300 budgeted group-by library (libagg.so).
 *
 * The operation (Section 3.1 of Wen, Borkar, Carey and Tsotras, "Revisiting
 * Aggregation for Data Intensive Applications: A Performance Study"): for every
 * distinct int64 grouping key among n input rows, one group record holding the
 * key and its bounded-state aggregates COUNT, SUM, MIN and MAX over the rows
 * with that key.  AVG is returned as the exact pair (SUM, COUNT).  All
 * aggregates are integers: COUNT is uint64, SUM is int64 taken modulo 2^64,
 * MIN and MAX are int64 (int32 input values are widened).
 *
 * The work runs under a strictly bounded working-memory budget given at
 * creation (Section 3.2: each query gets its own strict working-memory bound).
 * Groups that do not fit are partitioned, spilled to a staging area and
 * aggregated recursively, in the hybrid-hash style of Section 4.3 with the
 * Pre-Partitioning policy of Section 4.3.4 (the table is filled first; once it
 * is full, rows of resident groups aggregate in place and all other rows are
 * hash-partitioned and spilled).  A radix-sort + segmented-reduction path
 * (the Sort-based algorithm of Section 4.1) is available beside it.
 *
 * Conventions for every entry point:
 *  - Pointers named d_* are CUDA device pointers (or managed memory); h_* are
 *    host pointers.  Passing a host pointer where a device pointer is expected
 *    returns AGG_ERR_INVALID_ARG; there is no CPU fallback.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  agg_run only enqueues work; results are complete in stream
 *    order, and errors raised on the device are reported by agg_sync.
 *  - Input and output buffers are owned by the caller.  The library owns its
 *    working memory (inside the budget) and its staging area (outside it, as
 *    the paper's M excludes disk: Section 3.2, Section 4.1).
 *  - A handle is not thread-safe; distinct handles are independent.
 *  - Functions return AGG_OK or an agg_status error code; on error, output
 *    buffer contents are unspecified.
 */
#ifndef AGG_H
#define AGG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum agg_status {
  AGG_OK = 0,
  AGG_ERR_INVALID_ARG = 1,       /* NULL/host pointer, bad enum, bad size */
  AGG_ERR_BUDGET_TOO_SMALL = 2,  /* budget below AGG_MIN_BUDGET */
  AGG_ERR_OOM = 3,               /* cudaMalloc of working memory or staging failed */
  AGG_ERR_OUTPUT_CAPACITY = 4,   /* more groups than agg_output.capacity */
  AGG_ERR_STAGING_EXHAUSTED = 5, /* spill exceeded the reserved staging area */
  AGG_ERR_TIMEOUT = 6,           /* a bounded device-side wait gave up */
  AGG_ERR_CUDA = 7,              /* a CUDA runtime call failed */
  AGG_ERR_INTERNAL = 8           /* invariant violated (for example recursion depth) */
} agg_status;

/* Aggregate bitmask for agg_spec.ops (Section 3.1 bounded-state functions). */
enum { AGG_COUNT = 1u, AGG_SUM = 2u, AGG_MIN = 4u, AGG_MAX = 8u };

typedef enum agg_dtype { AGG_I32 = 0, AGG_I64 = 1 } agg_dtype;

/* AGG_PATH_HASH: Pre-Partitioning hybrid hash (Sections 4.3, 4.3.4).
 * AGG_PATH_SORT: radix sort + segmented reduction (Section 4.1); its output is
 * in ascending signed key order.
 * AGG_PATH_AUTO: each run takes the path the cost model predicts to be faster
 * (Section 5's models in bytes, Section 7's guidance): the input and result
 * bytes, the Pre-Partitioning spill R(1 - K/G) written and read back (Section
 * 5.3.4), the hash path's fall back to sorting when the groups are more than
 * 0.8 of the rows (Section 4.3), and the sort path's passes, each over a
 * bandwidth measured for that path on GB300.  Without an expected_groups hint
 * G is unknown and the hash path is taken.  Both paths share the handle's
 * working memory (a sort run leaves the table to be cleared before the next
 * hash run). */
typedef enum agg_path { AGG_PATH_HASH = 0, AGG_PATH_SORT = 1, AGG_PATH_AUTO = 2 } agg_path;

#define AGG_MIN_BUDGET ((size_t)1 << 20)
#define AGG_MAX_LEVELS 12

typedef struct agg_spec {
  uint32_t ops;             /* AGG_COUNT|AGG_SUM|AGG_MIN|AGG_MAX, non-zero */
  int32_t value_type;       /* agg_dtype of the input values */
  int32_t path;             /* agg_path */
  uint32_t flags;           /* reserved, must be 0 */
  uint64_t expected_groups; /* optional estimate of the result size G (Eq. 1); 0 = unknown */
  uint64_t seed;            /* hash seed of level 0; each level derives its own (Section 6.7) */
} agg_spec;

/* Knobs of the hash path; zero fields keep the defaults. */
typedef struct agg_tuning {
  double max_load_factor;  /* planned fill of a recursion round's table (default 0.5):
                              the round's slots are its records / max_load_factor; the
                              slot-table-size ratio of Section 6.7 is its inverse */
  uint32_t smem_entries;   /* per-block shared-memory pre-aggregation entries, power of
                              two 256..4096 (default 2048); 1 disables the cache */
  uint32_t fan_out;        /* spill partitions per level, power of two 16..256;
                              0 = planner (Eq. 1 with fudge factor, Section 4.3) */
  uint32_t warp_dedup;     /* warp-level combining of equal keys (__match_any_sync) before the
                              shared-memory table: 0 = default (off), 1 = on, 2 = off */
  uint32_t wait_limit_us;  /* limit of every bounded device-side wait (grid barriers), in
                              microseconds, at most 60,000,000 (60 s); 0 = 4 s.  A wait that
                              runs out ends the run with AGG_ERR_TIMEOUT (agg_sync) and the
                              handle is rebuilt */
  double fudge;            /* fudge factor F of Eq. 1 (default 1.2, Section 6.7) */
  uint32_t in_budget;      /* in-budget paths for inputs whose every group fits the table at once
                              (n at most half the slots): 0 = default (on), 2 = off (always the
                              spilling path).  Results do not depend on it */
  uint32_t sorted_input;   /* sorted-input path (Section 6.4: sort-based aggregation wins on sorted
                              data): a sampled order check, then one segmented reduction with no
                              table when the keys are non-decreasing.  0 = default (on), 2 = off.
                              Results do not depend on it */
  uint32_t max_levels;     /* recursion depth cap: records that reach this level are sorted and
                              reduced inside the run instead of partitioned again (Section 4.3's
                              fallback).  0 = default (the levels a sort-based split of 64-bit keys
                              by the fan-out's bits would need, at most AGG_MAX_LEVELS - 1), else
                              1..AGG_MAX_LEVELS - 1.  Results do not depend on it */
  uint32_t staging_tier;   /* where the spill staging lives (outside the budget, the paper's disk):
                              0 = default (device memory; pinned host memory, which the kernel
                              reaches over the host link, when device memory cannot be had),
                              1 = device memory only, 2 = host memory.  Results do not depend on it */
  uint32_t level0_slots;   /* slots of the level-0 table.  0 = default: at most AGG_LEVEL0_SLOTS.  A
                              table whose entries run far past L2 makes every update of a group that
                              is not hot a random read-modify-write in DRAM; with the cap the groups
                              that fill it first stay resident (Pre-Partitioning, Section 4.3.4) and
                              the rows of the others spill to level 1, whose rounds aggregate them in
                              shared memory.  1 = the whole table the budget gives (the paper's
                              sizing); else a cap of at least 4096 slots.  Results do not depend on it */
} agg_tuning;

#define AGG_LEVEL0_SLOTS 4194304u /* default cap of the level-0 table (2^22 slots) */

/* Output arrays, device pointers owned by the caller, one row per group.
 * Arrays of aggregates not in spec.ops may be NULL; keys must not be NULL.
 * capacity >= n always suffices. d_n_groups (optional) receives the group
 * count on the device when the run completes. */
typedef struct agg_output {
  int64_t* keys;
  uint64_t* count;
  int64_t* sum;
  int64_t* min;
  int64_t* max;
  uint64_t capacity;
  uint64_t* d_n_groups;
} agg_output;

/* Counters of the last completed run (agg_get_stats). */
typedef struct agg_stats {
  uint64_t n_rows;
  uint64_t n_groups;
  uint64_t levels;                               /* recursion levels used (1 = no spill) */
  uint64_t rounds;                               /* table rounds over all levels */
  uint64_t spill_records[AGG_MAX_LEVELS];        /* records spilled by level L */
  uint64_t resident_groups[AGG_MAX_LEVELS];      /* groups completed at level L */
  uint64_t spill_bytes_written;                  /* 16 B per spilled record */
  uint64_t spill_bytes_read;
  uint64_t rows_at_full;                         /* first level-0 row of a tile that spilled (~R_H) */
  uint64_t table_slots;
  uint64_t table_capacity;                       /* planned groups per table, max_load_factor * slots (K) */
  uint64_t table_bytes;                          /* working memory used inside the budget */
  uint64_t budget_bytes;
  uint64_t staging_bytes;                        /* reserved staging (outside the budget) */
  uint64_t fan_out;
  uint64_t status_bits;                          /* 1 << agg_status of device-side errors seen */
  uint64_t kernel_launches;                      /* kernels this handle has launched, cumulative */
  uint64_t phase_ns[12];                         /* hash path, block 0's time per phase: level-0 pass,
                                                    barrier wait, level-0 emit, partition lists, round
                                                    aggregation, barrier waits, round emit, total,
                                                    shared-memory rounds: count, scatter, aggregate */
  uint64_t sorted_input;                         /* 1 when the run took the sorted-input path */
  uint64_t fallback_records;                     /* records the recursion fallback sorted (0 = none) */
  uint64_t fallback_level;                       /* the level at which it ran */
  uint64_t staging_in_host;                      /* 1 when the staging area is in host memory */
  uint64_t path;                                 /* path of the last run: AGG_PATH_HASH or AGG_PATH_SORT */
} agg_stats;

/* Planner output (host-only arithmetic, no GPU needed). */
typedef struct agg_plan_info {
  uint64_t entry_bytes;     /* bytes per table slot entry (32 or 64) */
  uint64_t table_slots;     /* slots S of the table inside the budget */
  uint64_t table_capacity;  /* K = floor(max_load_factor * S) */
  uint64_t fan_out;         /* spill partitions per level */
  uint64_t active_slots;    /* slots used at level 0 for this n */
  uint64_t working_bytes;   /* bytes of the budget in use */
  uint64_t staging_bytes;   /* staging reserved for n rows */
  uint64_t in_budget_path;  /* path agg_run takes for n rows: 0 = spilling hybrid hash, 1 = in-budget,
                               partitioned into shared-memory tables (small n), 2 = in-budget, one
                               table probed linearly (n at most half the slots) */
  uint64_t partitions;      /* partitions of path 1 (else 0) */
  double hash_bytes;        /* cost model: predicted DRAM bytes of the hash path for n rows */
  double sort_bytes;        /* and of the sort path */
  double hash_seconds;      /* predicted run times (bytes over each path's measured bandwidth, plus */
  double sort_seconds;      /* its fixed launch cost) */
  uint64_t chosen_path;     /* the path an AGG_PATH_AUTO run of n rows takes (AGG_PATH_HASH or _SORT) */
} agg_plan_info;

typedef struct agg_handle agg_handle;

/* Creates a group-by handle: validates spec, allocates the working memory
 * (hash table, tags, control block) inside memory_budget_bytes on the current
 * device and clears it.  Errors: AGG_ERR_INVALID_ARG (NULL out/spec, bad ops,
 * value_type or path, flags != 0), AGG_ERR_BUDGET_TOO_SMALL, AGG_ERR_OOM,
 * AGG_ERR_CUDA.  On success *out owns the memory until agg_destroy. */
agg_status agg_create(size_t memory_budget_bytes, const agg_spec* spec, agg_handle** out);

/* Replaces the tuning knobs (Section 6.7 slot ratio and fudge factor, fan-out,
 * shared-memory pre-aggregation size, warp dedup).  Results do not depend on
 * tuning.  Errors: AGG_ERR_INVALID_ARG for out-of-range values. */
agg_status agg_set_tuning(agg_handle* h, const agg_tuning* t);

/* Reserves the staging area for inputs of up to max_rows rows, so that a later
 * agg_run with n <= max_rows allocates nothing (and may be captured in a CUDA
 * graph).  Errors: AGG_ERR_OOM, AGG_ERR_CUDA. */
agg_status agg_reserve(agg_handle* h, uint64_t max_rows);

/* Enqueues the group-by of n rows on `stream`.  d_keys: n int64 keys; d_vals:
 * n values of spec.value_type (may be NULL when ops == AGG_COUNT).  Both must
 * stay valid until the stream reaches the end of the run.  Writes the groups to
 * `out` in unspecified order (hash path) or ascending key order (sort path) and
 * the group count to out->d_n_groups.  May call cudaMalloc to grow the staging
 * area when n exceeds the last reservation (not allowed during stream capture:
 * AGG_ERR_INVALID_ARG).  Host-side errors are returned; device-side errors
 * (output capacity, staging exhausted, timeouts) surface in agg_sync. */
agg_status agg_run(agg_handle* h, const int64_t* d_keys, const void* d_vals, uint64_t n,
                   const agg_output* out, void* stream);

/* Same group-by on host buffers; writes the n_groups result rows into the host
 * arrays of h_out (capacity counted in rows) and *n_groups.  Synchronous.
 * Hash path, when the device can address every buffer (pinned memory, or
 * pageable memory on a host with coherent device access such as Grace over
 * NVLink-C2C): the kernel reads the input from host memory and writes the
 * result rows straight into h_out, so that both transfers overlap its work.
 * Otherwise (and on the sort path) the input is copied to device buffers owned
 * by the handle and the result is copied back after the run; pinned host memory
 * gives the full copy bandwidth.  Errors as agg_run and agg_sync;
 * AGG_ERR_OUTPUT_CAPACITY when n_groups exceeds h_out->capacity. */
agg_status agg_run_host(agg_handle* h, const int64_t* h_keys, const void* h_vals, uint64_t n,
                        const agg_output* h_out, uint64_t* n_groups, void* stream);

/* Waits for the last run of h, returns its device-side status and stores the
 * group count in *n_groups_host (may be NULL).  Clears the device status. */
agg_status agg_sync(agg_handle* h, uint64_t* n_groups_host);

/* Copies the counters of the last run (waits for it). */
agg_status agg_get_stats(agg_handle* h, agg_stats* s);

/* Releases every allocation of h (waits for its work first).  NULL is allowed. */
agg_status agg_destroy(agg_handle* h);

/* Static description of a status code. */
const char* agg_strerror(agg_status s);

/* ---- Batched form: many independent group-bys in one persistent launch ---- */

/* One instance of a batch: its input, its working-memory budget and its output
 * (device pointers, caller-owned; out.d_n_groups is ignored: the counts are
 * returned by agg_batch_sync). */
typedef struct agg_batch_item {
  const int64_t* d_keys;
  const void* d_vals;
  uint64_t n;
  size_t budget;            /* this instance's budget, >= AGG_MIN_BUDGET */
  uint64_t expected_groups; /* optional estimate of its result size; 0 = unknown */
  agg_output out;
} agg_batch_item;

/* Knobs of the batch; zero fields keep the defaults (or the tuning table). */
typedef struct agg_batch_tuning {
  uint32_t team_blocks;    /* thread blocks that run one instance together (power of two) */
  uint32_t smem_entries;   /* shared-memory table entries per block (power of two, >= 512) */
  double max_load_factor;
  uint32_t fan_out;
  uint32_t use_graph;      /* 0 = default (capture the launch in a CUDA graph), 2 = launch directly */
} agg_batch_tuning;

typedef struct agg_batch agg_batch;

/* Plans a batch of `count` instances sharing spec.ops and spec.value_type
 * (spec.path must be AGG_PATH_HASH): instances are assigned to teams of thread
 * blocks longest-first; every team owns working memory large enough for the
 * largest budget among its instances (each instance uses at most its own
 * budget of it, one instance at a time) and staging for those that may spill.
 * Allocates everything the runs need.  Errors: AGG_ERR_INVALID_ARG (also an
 * item whose input or output arrays are not device memory, whose values are
 * missing while SUM, MIN or MAX is asked for, or whose keys or values are not
 * aligned to their element size), AGG_ERR_BUDGET_TOO_SMALL (an item's budget),
 * AGG_ERR_OOM, AGG_ERR_CUDA. */
agg_status agg_batch_create(const agg_spec* spec, const agg_batch_item* items, uint32_t count,
                            const agg_batch_tuning* t, agg_batch** out);

/* Runs every instance of the batch with one cooperative kernel launch (replayed
 * from a CUDA graph captured on the first run), asynchronously on `stream`. */
agg_status agg_batch_run(agg_batch* b, void* stream);

/* Waits for the last run; stores each instance's group count in n_groups[i]
 * (host array of `count` entries, may be NULL) and returns the first device-side
 * error of any instance. */
agg_status agg_batch_sync(agg_batch* b, uint64_t* n_groups);

/* Releases the batch (waits for its work first).  NULL is allowed. */
agg_status agg_batch_destroy(agg_batch* b);

/* ---- Served form: queries arrive over time and share the device ---- */

/* One query submitted to a server: input, declared budget and output (device
 * pointers, caller-owned, valid until the query completes).  If `ready` is a
 * cudaEvent_t (may be NULL), the query's work waits for it (for example the
 * event recorded after the input was produced). */
typedef struct agg_query {
  const int64_t* d_keys;
  const void* d_vals;
  uint64_t n;
  size_t budget;            /* declared working-memory budget, >= AGG_MIN_BUDGET */
  uint64_t expected_groups; /* optional */
  agg_output out;           /* out.d_n_groups is ignored: see agg_server_poll */
  void* ready;
} agg_query;

enum { AGG_QUERY_QUEUED = 0, AGG_QUERY_RUNNING = 1, AGG_QUERY_DONE = 2, AGG_QUERY_FAILED = 3 };

typedef struct agg_query_info {
  int32_t state;        /* AGG_QUERY_* */
  int32_t status;       /* agg_status of a finished query */
  uint64_t n_groups;
  double t_submit;      /* host steady-clock seconds */
  double t_start;       /* admitted and launched */
  double t_done;        /* completion observed by agg_server_progress */
  uint32_t team_blocks; /* thread blocks that ran it (0: ordinary launches, no cooperative team) */
  uint32_t path;        /* AGG_PATH_HASH or AGG_PATH_SORT (an AGG_PATH_AUTO server chooses per query) */
} agg_query_info;

typedef struct agg_server_stats {
  uint64_t submitted, completed, running, queued;
  uint64_t pool_bytes, pool_in_use, pool_peak;  /* working memory of admitted queries */
  uint64_t max_concurrent;                      /* most queries running at once */
  uint64_t staging_bytes, staging_in_use, staging_peak;  /* staging pool of queries that may spill */
  uint64_t blocks, blocks_in_use;               /* co-resident thread blocks, and those held by running queries */
} agg_server_stats;

/* Smallest staging pool of a server (see agg_server_create). */
#define AGG_SERVER_MIN_STAGING ((size_t)1 << 30)

typedef struct agg_server agg_server;

/* Creates a server with a device memory pool of pool_bytes for the working
 * memory of its queries (their declared budgets, the multi-user memory
 * constraint of Section 3.2) and at most max_active queries running at once.
 * Beside it, in the same allocation, the server keeps a staging pool of
 * max(pool_bytes / 2, AGG_SERVER_MIN_STAGING) bytes for the spill staging of
 * the queries that may spill (outside their budgets, as the paper's M excludes
 * disk).  Nothing else is allocated while queries run.
 * spec.ops and spec.value_type apply to every query. */
agg_status agg_server_create(const agg_spec* spec, size_t pool_bytes, uint32_t max_active, agg_server** out);

/* Queues a query (never blocks, never launches).  *ticket identifies it.
 * AGG_ERR_INVALID_ARG when its arrays are not device memory, its values are
 * missing while SUM, MIN or MAX is asked for, its keys or values are not aligned
 * to their element size, its budget exceeds the pool, or its staging could not
 * fit the staging pool; nothing is queued then. */
agg_status agg_server_submit(agg_server* s, const agg_query* q, uint64_t* ticket);

/* One turn of the request loop: notices finished queries (freeing their
 * budget, staging, thread blocks and slot), then admits queued queries in
 * arrival order, each launched at once on its slot's stream so that admitted
 * queries run concurrently.  A query is admitted when a slot is free, its
 * declared budget fits the free pool, its staging (if it may spill) fits the
 * staging pool, and enough thread blocks are free: the teams of running queries
 * never add up to more blocks than the GPU holds at once, so their cooperative
 * grids never wait on one another.  A query whose groups all fit its table at
 * once (n at most half its slots) runs on the in-budget kernels, ordinary
 * launches that hold no team; so does a query an AGG_PATH_AUTO server sends to
 * the sort path (only when one sort round holds it).  Any other query wants
 * about one block per 8k rows (a power of two, 8 to the whole GPU) and gets
 * fewer when fewer are free (at least 8, or all it wants if less), or when its
 * staging (one open chunk per block and partition) would not fit the staging
 * pool.  Queries wanting more than 32 blocks share all but a quarter of the
 * blocks, which stays free for the small ones; such a query waiting for blocks
 * does not hold back the smaller queries behind it, while one waiting for
 * memory holds back every later query.  Non-blocking.  *completed (may be NULL)
 * receives the number of queries finished now. */
agg_status agg_server_progress(agg_server* s, uint32_t* completed);

/* State, result size and timestamps of a query. */
agg_status agg_server_poll(agg_server* s, uint64_t ticket, agg_query_info* info);

agg_status agg_server_get_stats(agg_server* s, agg_server_stats* st);

/* Waits for every running query, then releases the server. */
agg_status agg_server_destroy(agg_server* s);

/* Size of the fixed working memory of agg_run_noalloc. */
#define AGG_NOALLOC_SLOTS (1u << 18)
#define AGG_NOALLOC_MAX_ROWS ((uint64_t)AGG_NOALLOC_SLOTS / 4)

/* The in-budget hash group-by for callers that cannot allocate device memory.
 * The paper has no counterpart: it is an addition for callers that may not
 * call cudaMalloc or cudaFree at all, such as code running inside a framework
 * that owns every device allocation, or code on a latency-critical path that
 * cannot afford an allocation or the device-wide synchronisation of a free.
 * Nothing is allocated: the working memory (about 17 MB: control block, tag
 * bytes and AGG_NOALLOC_SLOTS table entries) is a file-scope __device__ array
 * of libagg.so that every GPU loading the library holds until the process
 * exits.  n may be at most AGG_NOALLOC_MAX_ROWS, a quarter of the slots (else
 * AGG_ERR_INVALID_ARG, and nothing runs).  The run uses the in-budget path of
 * agg_run for small inputs: rows are split by hash into partitions that thread
 * blocks aggregate in shared memory, and a key that does not fit there probes
 * linearly across the table's slots, so every group is resident whatever the
 * keys' hashes (key sets built to collide included), and no staging area is
 * ever needed.
 * spec: as for agg_create, with path AGG_PATH_HASH.  d_keys, d_vals, out: as
 * for agg_run (device pointers, caller-owned).  The call enqueues the work on
 * `stream`, reads the status and group count back in stream order, waits for
 * them, and returns the run's status (AGG_ERR_OUTPUT_CAPACITY when the groups
 * exceed out->capacity), with the group count in *n_groups (may be NULL).  The
 * first call on a device sets that device up (it looks up the array's device
 * address and the kernels' launch shape), so make it before any stream
 * capture.  Every call shares the one array and clears the part it uses first:
 * calls whose work overlaps on the GPU (other streams, other threads) race on
 * it and must be serialised by the caller. */
agg_status agg_run_noalloc(const agg_spec* spec, const int64_t* d_keys, const void* d_vals, uint64_t n,
                           const agg_output* out, uint64_t* n_groups, void* stream);

/* Host-only planning: the table size, capacity and fan-out agg_create/agg_run
 * would choose for this budget, spec and n (Eq. 1 adapted to bytes, Section
 * 4.3).  No GPU is touched.  Errors: AGG_ERR_INVALID_ARG,
 * AGG_ERR_BUDGET_TOO_SMALL. */
agg_status agg_plan(size_t memory_budget_bytes, const agg_spec* spec, const agg_tuning* t, uint64_t n,
                    agg_plan_info* out);

#ifdef __cplusplus
}
#endif

#endif /* AGG_H */
