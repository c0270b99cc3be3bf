/* ht.h -- C ABI of a GPU hash set/map for state-space exploration (sm_103a).
 *
 * The operations follow the problem statement of Cassee & Wijs, "Analysing
 * the Performance of GPU Hash Tables for State Space Exploration" (GaM 2017):
 *
 *   Section 5      "find, else insert": for every element of a sequence,
 *                  look it up; if found do nothing, otherwise insert it.
 *   Section 4.1    Cuckoo hashing (Alcantara et al.): k hash functions,
 *                  eviction chains, a stash, rebuild with new constants.
 *   Section 4.2    The GPUexplore bucket table: hash to a bucket of slots
 *                  read cooperatively by a group of lanes, atomic claim of a
 *                  free slot, the next hash function when a bucket is full.
 *   Section 3.2    BFS over state vectors with open/closed sets kept in the
 *                  hash table.
 *
 * Conventions for every call
 * --------------------------
 *  * Pointers named d_* are DEVICE pointers owned by the caller; h_* are host
 *    pointers owned by the caller.  Nothing keeps a caller pointer after the
 *    call returns, except that the work it enqueued reads/writes it later in
 *    stream order.
 *  * `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls are
 *    stream-ordered and asynchronous unless they say "synchronises".
 *  * Operations on one table must be issued in order on one stream at a time.
 *    Different tables are independent.
 *  * Keys: key_width 32 -> uint32 keys, 0xFFFFFFFF reserved (empty marker);
 *    key_width 64 -> uint64 keys whose top bit must be 0; key_width 128 ->
 *    (low, high) uint64 pairs, bit 63 of the high word reserved; key_width
 *    192..512 -> rows of key_width/64 uint64 words, no value reserved (see
 *    ht_create).  A reserved key in a batch is skipped (is_new/found = 0) and
 *    makes the next synchronising call on the table return HT_ERR_INVALID;
 *    the rest of the batch is processed.
 *  * Values (maps): only tables with key_width 32 carry a uint32 value, packed
 *    with the key in one 64-bit slot so that a slot moves atomically.
 *  * Table memory is allocated by ht_create and freed by ht_destroy.
 *  * Errors found on the device (reserved key, table full) are sticky and are
 *    reported by the next synchronising call (ht_sync, ht_size, ht_export).
 *    HT_ERR_CUDA is returned when a CUDA call or launch fails.
 */
#ifndef HT_H_
#define HT_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { HT_BUCKET = 0, HT_CUCKOO = 1 } ht_scheme;

typedef enum {
    HT_OK = 0,
    HT_ERR_INVALID = 1,  /* bad argument, or a reserved key was seen */
    HT_ERR_OOM = 2,      /* device allocation failed */
    HT_ERR_FULL = 3,     /* keys could not be placed even after rebuilds */
    HT_ERR_CUDA = 4,     /* a CUDA call or kernel launch failed */
    HT_ERR_TIMEOUT = 5   /* a bounded device wait gave up */
} ht_status;

/* Tunables.  A zero field means "default".  Section 5 of the paper fixes a
 * table of 1.25x the unique keys (load 0.8) and about four hash functions;
 * the defaults below are chosen for that load on large tables:
 *   num_hashes     bucket: 16 (hashes are computed lazily, a later one only
 *                  when the earlier buckets are full); cuckoo: 4.  Max 16 /
 *                  8 respectively.
 *   max_evictions  cuckoo eviction-chain bound, default 256, max 4096.
 *   stash_slots    default 101 (both schemes).
 *   bucket_slots   8, 16 or 32 slots of 8 bytes; default 16 (128 bytes).
 *   lanes_per_key  lanes that read one bucket (2..32, with 1 to 8 slots per
 *                  lane); default 2 (measured fastest on GB300: fewer lanes
 *                  per key spread each round's fixed cost over more keys).
 *   max_rebuilds   rebuild attempts with fresh hash constants, default 8.
 *   max_batch      cuckoo keys per probe/insert launch pair (sizes the
 *                  in-batch dedup scratch), default 2^22.
 *   seed           hash-constant seed.
 *   l2_persist     1: launches on this table carry an L2 access-policy
 *                  window marking the slot array persisting when it fits
 *                  the device's persisting L2 (else, for Cuckoo, the dedup
 *                  claim set); this raises the process's persisting L2
 *                  set-aside (cudaLimitPersistingL2CacheSize), which stays
 *                  reserved after the table is destroyed.  Default: 0.
 *   grow_load_permille  0 (default): fixed capacity.  Else a synchronising
 *                  call (ht_sync, ht_size, ht_export) that finds
 *                  the table above this load (per mille of its slots), or
 *                  using its overflow set, doubles its capacity (ht_grow)
 *                  until it is below (100..1000; 0 = off).  Between two
 *                  synchronising calls the keys still have to fit the table,
 *                  stash and overflow set as they are.
 *   digest_bits    keys wider than 128 bits only: 0 (default) or 64 keeps
 *                  the whole 64-bit key digest; 1..63 keeps only its low
 *                  bits, so that distinct keys share digests.  A test knob:
 *                  it makes the full-key comparisons that tell such keys
 *                  apart run often (results are unchanged; placement gets
 *                  worse).  Other key widths: must be 0.
 *   cuckoo_chain_h1  Cuckoo: 0 (default) inserts a new key at the first of
 *                  its slots h_1..h_k that its probe saw empty -- for keys of
 *                  up to 128 bits the probe stores it there with a CAS from
 *                  EMPTY (in slot order when another key took the slot
 *                  first) and only a key whose k slots were all full runs an
 *                  eviction chain, from h_1; for longer keys the chain
 *                  starts at that slot.  1 keeps Section 4.1's rule: an
 *                  insertion starts at h_1 (a CAS there only when h_1 was
 *                  empty, otherwise an eviction chain from h_1).  Both keep
 *                  "a key stored at h_j has h_1 .. h_(j-1) occupied" (slots
 *                  never become empty again), so results are the same; the
 *                  default makes fewer atomics.
 *   publish_wait_polls  keys wider than 128 bits, bucket scheme: how many
 *                  times a reader polls a claimed, unpublished slot header
 *                  of its key's tag (with back-off) before it gives up and
 *                  the table reports HT_ERR_TIMEOUT; 0 = default 2^20 (about
 *                  0.1 s).  Tests set it small.  */
typedef struct ht_params {
    uint32_t num_hashes;
    uint32_t max_evictions;
    uint32_t stash_slots;
    uint32_t bucket_slots;
    uint32_t lanes_per_key;
    uint32_t max_rebuilds;
    uint64_t max_batch;
    uint64_t seed;
    int32_t l2_persist;
    uint32_t grow_load_permille;
    uint32_t digest_bits;
    uint32_t cuckoo_chain_h1;
    uint32_t publish_wait_polls;
    uint32_t reserved_;
} ht_params;

typedef struct ht_table ht_table;

/* Fills *p with the defaults of `scheme`.  Host only. */
ht_status ht_default_params(ht_scheme scheme, ht_params* p);

/* Creates an empty table of at least `capacity` slots (rounded up to whole
 * buckets, for both schemes) on the current device.  Section 5: the paper
 * sizes the table at 1.25x the number of unique keys.  params may be NULL.
 * Allocates the slot array, stash, overflow set and counters (and, for
 * Cuckoo, the dedup scratch) in the order of `stream` (cudaMallocAsync) and
 * clears them on `stream`; use the table on other streams only after work
 * on `stream` is ordered before that use.
 * key_width 32, 64 or 128: 128-bit keys are two 64-bit words (low word
 * first, 16-byte aligned, bit 63 of the high word reserved) for state
 * vectors wider than 64 bits, in 16-byte slots written with 16-byte atomics
 * (compare-and-swap claims, exchange evictions for Cuckoo); bucket scheme:
 * buckets of 8 slots (bucket_slots must be 8, lanes_per_key 2 or 4; with
 * params NULL: 8 and 2); no stash (the overflow set takes what does not
 * fit), no values.  128-bit tables support find-or-put (with append),
 * insert without values, lookup without values, export, size, clear, grow,
 * stats, ht_successors and ht_bfs over models up to 127 bits wide (not
 * ht_bfs_fused or the batched forms).
 * key_width 192, 256, ..., 512 (W = key_width / 64 words, 3..8): long keys
 * (multi-word state vectors; Sections 3.2 and 4.2 for GPUexplore's vectors,
 * Section 7 for Cuckoo hashing of keys of any length).  A key is W uint64
 * words, one key per row of the caller's array (row-major n x W, 8-byte
 * aligned); no value is reserved.  No atomic covers a whole key, so the
 * words sit in a key store beside the slots: bucket scheme -- one 8-byte
 * header per slot, 16 to a 128-byte bucket (bucket_slots must be 16;
 * lanes_per_key unused), claimed with a compare-and-swap and published with
 * a release store after the key's words are written (a reader that meets a
 * claimed, unpublished header of its tag waits, bounded; HT_ERR_TIMEOUT if
 * the bound is hit); Cuckoo -- 16-byte (digest, row) entries moved by
 * eviction chains, the words written once to their row, no stash.  Long-key
 * tables support find-or-put, insert and lookup without values or append,
 * export (rows of W words), size, clear, grow and stats; not ht_bfs,
 * ht_successors, the batched forms or ht_multi_find_or_put.
 * Errors: HT_ERR_INVALID (capacity 0 or > 2^40, key_width not one of the
 * above, bad params), HT_ERR_OOM, HT_ERR_CUDA.  *out is NULL on error. */
ht_status ht_create(uint64_t capacity, ht_scheme scheme, uint32_t key_width,
                    const ht_params* params, void* stream, ht_table** out);

/* Frees the table (synchronises the device).  NULL is accepted. */
ht_status ht_destroy(ht_table* t);

/* Batched find-or-put (Section 5): for each key, insert it if it is absent.
 * d_keys: n keys (uint32 or uint64 by key_width).  d_is_new (nullable): n
 * bytes, 1 where this call stored the key.  Among equal keys of one batch
 * exactly one is flagged (which one is unspecified).  On a map the stored
 * value is 0. */
ht_status ht_find_or_put(ht_table* t, const void* d_keys, uint64_t n,
                         uint8_t* d_is_new, void* stream);

/* find-or-put that also appends each newly stored key to d_new_keys at
 * positions reserved by atomically adding to *d_new_count (a device uint64
 * counter the caller zeroes; the call does not reset it).  d_new_keys must
 * have room for every key of the batch plus *d_new_count.  Used to turn a
 * BFS level's successors into the next frontier (Section 3.2's open set). */
ht_status ht_find_or_put_append(ht_table* t, const void* d_keys, uint64_t n,
                                uint8_t* d_is_new, void* d_new_keys,
                                unsigned long long* d_new_count, void* stream);

/* Insert-if-absent with values (key_width 32 maps; d_values must be NULL for
 * key_width 64): Section 5's find-or-insert applied to (key, value) pairs,
 * where a key that is found is left as it is, and Section 5.1.1's rule that
 * a duplicate must not be stored twice.  A key already present keeps its
 * value; among equal keys in one batch one of the supplied values wins.
 * d_keys, d_values: n device words owned by the caller.  Asynchronous on
 * `stream`; reserved keys and a full table are reported by the next
 * synchronising call (ht_sync, ht_size). */
ht_status ht_insert(ht_table* t, const void* d_keys, const uint32_t* d_values,
                    uint64_t n, void* stream);

/* Lookup (Section 4.1: at most k slots; Section 4.2: at most k buckets).
 * d_found (nullable): n bytes, 1 if present.  d_values (nullable, maps only):
 * n uint32, the stored value or 0. */
ht_status ht_lookup(ht_table* t, const void* d_keys, uint64_t n,
                    uint32_t* d_values, uint8_t* d_found, void* stream);

/* Synchronises `stream`, runs a pending rebuild (Section 4.1: when the stash
 * is full and an insertion fails, rebuild with new hash constants) and
 * returns the table's sticky status. */
ht_status ht_sync(ht_table* t, void* stream);

/* Number of stored keys (synchronises; runs ht_sync first). */
ht_status ht_size(ht_table* t, uint64_t* out, void* stream);

/* Copies every stored key (and value, if d_values_out is non-NULL) into the
 * caller's buffers of `cap` entries, in unspecified order; *count = number of
 * stored keys (synchronises).  An entry is a key in the table's input layout:
 * one uint32/uint64, a 16-byte (low, high) pair for 128-bit keys, or a row of
 * W words for long keys.  HT_ERR_INVALID if cap < count (nothing is
 * guaranteed about the buffers then). */
ht_status ht_export(ht_table* t, void* d_keys_out, uint32_t* d_values_out,
                    uint64_t cap, uint64_t* count, void* stream);

/* Empties the table, keeping its capacity and hash constants. */
ht_status ht_clear(ht_table* t, void* stream);

/* Moves the table to `new_capacity` slots (rounded up to whole buckets):
 * every stored key (and value) is copied out of the table, stash and
 * overflow set and inserted into new storage with the current hash
 * constants; the old storage is freed.  Synchronises `stream`.  Not part of
 * the paper (Sections 4.1, 4.2 report a full table); it lets a table start
 * small.  HT_ERR_INVALID if new_capacity is 0 or too large; HT_ERR_FULL if
 * the keys do not fit the new capacity (the table is then unchanged);
 * HT_ERR_OOM if the new storage cannot be allocated (unchanged too).  The
 * table must not be in use on another stream meanwhile. */
ht_status ht_grow(ht_table* t, uint64_t new_capacity, void* stream);

/* Table facts: slots, hash functions, rebuilds done so far. */
ht_status ht_info(const ht_table* t, uint64_t* slots, uint32_t* num_hashes,
                  uint32_t* rebuilds);

/* Counters of a table since its last clear (ht_clear), rebuild or growth:
 * what the paper's analysis turns on -- stored keys, the stash and rebuilds
 * of Section 4.1, Cuckoo's eviction work (Section 4.1: chain length grows
 * with the load) -- read from the device. */
typedef struct ht_table_stats {
    uint64_t size;            /* keys stored (table + stash + overflow set) */
    uint64_t dropped;         /* keys that found no place (then HT_ERR_FULL) */
    uint64_t exchanges;       /* Cuckoo: atomic exchanges made by insertion
                                 chains (Section 4.1; for 32/64-bit keys only
                                 keys that found all k slots full run one);
                                 0 for the bucket scheme */
    uint32_t stash_used;      /* stash slots in use */
    uint32_t overflow_used;   /* overflow-set slots in use */
    uint32_t rebuilds;        /* rebuilds since ht_create */
    uint32_t flags;           /* device status bits: 1 reserved key seen,
                                 2 rebuild pending, 4 key dropped */
    uint64_t probes;          /* Cuckoo: slots read by find-or-put and lookup
                                 probes (h_1, then h_2..h_k when h_1 is occupied);
                                 0 for the bucket scheme (a per-key count there
                                 would put one shared counter on the hot path)
                                 and for 128-bit tables */
    uint64_t probe_misses;    /* Cuckoo (32/64-bit keys): keys that find-or-put
                                 and insert found nowhere (absent from the
                                 table; lookups are not counted) ... */
    uint64_t probe_miss_reads;/* ... and the slots their probes read (h_1,
                                 then h_2.. up to the first empty slot) */
    uint64_t probe_cas;       /* Cuckoo (32/64/128-bit keys): compare-and-swaps of
                                 absent keys into the first empty slot their
                                 probe saw (and on, in slot order, when another
                                 key took it first); with exchanges, every
                                 atomic an insertion made in the table */
} ht_table_stats;

/* Reads the table's counters into *out (caller-owned host memory);
 * synchronises `stream`; changes nothing (no rebuild or growth runs).
 * HT_ERR_INVALID for a NULL table or out; HT_ERR_CUDA if the copy fails. */
ht_status ht_stats(ht_table* t, ht_table_stats* out, void* stream);

const char* ht_status_str(ht_status s);

/* ---------------------------------------------------------------------------
 * Frontier compaction (the BFS open set, Section 3.2): appends d_keys[i] for
 * every i with d_flags[i] != 0 to d_out at positions reserved on the device
 * counter *d_count (not reset by the call).  Order is unspecified.
 * ------------------------------------------------------------------------- */
ht_status ht_compact(const void* d_keys, const uint8_t* d_flags, uint64_t n,
                     uint32_t key_width, void* d_out, unsigned long long* d_count,
                     void* stream);

/* ---------------------------------------------------------------------------
 * State-space exploration (Section 3.2: a model is a set of finite-state
 * processes in parallel composition; BFS from the vector of initial local
 * states keeps the open and closed sets in the hash table; successor vectors
 * are built from each process's enabled transitions).
 *
 * Model layout (host struct, copied to the device by each call):
 *   component c < num_components (<= 16) has local states stored in bits[c]
 *   bits, packed LSB-first: c occupies bits [o_c, o_c + bits[c]) with
 *   o_c = bits[0] + ... + bits[c-1]; the packed vector must fit the table's
 *   key width (<= 31 bits for 32-bit keys, <= 63 for 64-bit keys).
 *   Local state u (< 32) of component c has deg[c][u] (<= 4) transitions j
 *   to tgt[c][u][j] with label lab[c][u][j]: 0 = local action, p+1 = member
 *   of synchronising pair p = (pair_c1[p], pair_c2[p]), p < num_pairs <= 8.
 * Successors of a state s: for every component c and every label-0
 * transition of c at s_c, s with s_c replaced by its target; for every pair
 * p and every combination of a label-(p+1) transition of pair_c1[p] at its
 * local state and one of pair_c2[p] at its local state, s with both local
 * states replaced.  Labelled transitions never fire alone.
 * ------------------------------------------------------------------------- */
typedef struct ht_model {
    int32_t num_components;
    int32_t num_pairs;
    uint8_t bits[16];
    uint8_t pair_c1[8];
    uint8_t pair_c2[8];
    uint8_t deg[16][32];
    uint8_t tgt[16][32][4];
    uint8_t lab[16][32][4];
} ht_model;

/* Writes the successors of n states (key_width-bit vectors) to d_succ at
 * positions reserved on the device counter *d_count (not reset; order
 * unspecified).  HT_ERR_INVALID for a malformed model.  If more than `cap`
 * successors would be written, the excess is not written and *d_count still
 * counts them, so the caller can detect it (cap >= n * the model's largest
 * per-state successor count never overflows). */
ht_status ht_successors(const ht_model* h_model, uint32_t key_width, const void* d_states,
                        uint64_t n, void* d_succ, uint64_t cap,
                        unsigned long long* d_count, void* stream);

typedef struct ht_bfs_result {
    uint64_t levels;        /* non-empty BFS levels */
    uint64_t states;        /* reachable states stored */
    uint64_t successors;    /* successor vectors generated (with repeats) */
    int32_t complete;       /* 1 if the exploration finished within the limits */
    int32_t reserved_;
} ht_bfs_result;

/* Level-synchronous BFS from state s0 over `model`, with the table `t` as the
 * set of visited states (it should be empty; every reachable state is
 * find-or-put into it once per generating transition).  Each level: generate
 * the successors of the frontier, find-or-put them, and the new ones (the
 * is_new keys) become the next frontier.  d_states (nullable, key_width-bit
 * entries, states_cap of them) receives every reachable state in level
 * order: level d occupies [sum of sizes of levels < d, + size of level d).
 * h_level_sizes (nullable, max_levels entries) receives the level sizes.
 * Stops when a level is empty (complete = 1), or when max_levels or
 * states_cap would be exceeded (complete = 0).  Synchronises once per level.
 * With a 128-bit table (models wider than 63 bits) states are 16-byte
 * pairs (low word first) and s0 is the initial state's low word (its high
 * word is 0).
 * Allocates its work buffers with cudaMalloc and frees them before
 * returning. */
ht_status ht_bfs(ht_table* t, const ht_model* h_model, uint64_t s0, uint32_t max_levels,
                 uint64_t* h_level_sizes, void* d_states, uint64_t states_cap,
                 ht_bfs_result* result, void* stream);

/* ht_bfs with each level's successor generation and find-or-put fused into
 * one launch (exploration on the fly, as GPUexplore does, Section 3.2):
 * a warp generates its frontier states' successors into shared memory and
 * finds-or-puts them from there, so no successor buffer goes through device
 * memory.  Bucket-scheme tables only (HT_ERR_INVALID for Cuckoo, whose
 * find-or-put needs two launches); same arguments, results and errors as
 * ht_bfs. */
ht_status ht_bfs_fused(ht_table* t, const ht_model* h_model, uint64_t s0, uint32_t max_levels,
                       uint64_t* h_level_sizes, void* d_states, uint64_t states_cap, ht_bfs_result* result,
                       void* stream);

/* ---------------------------------------------------------------------------
 * Batched find-or-put over many tables in one call (the batched form of
 * Section 5's find-or-insert, for workloads with many small tables).  Item i
 * runs find-or-put of h_list[i].n keys (device memory, the key width of
 * tables[h_list[i].table]) and writes is_new to h_list[i].d_is_new (device,
 * nullable).  Bucket-scheme items with the same key width and bucket shape
 * run together in one launch, one 32-key tile per warp against its own
 * table; Cuckoo items run one after another in list order.  Items that name
 * the same table behave as one batch: a key new to the table is flagged new
 * in exactly one of its occurrences across them.  Asynchronous on `stream`;
 * every table must be used on this stream only meanwhile.  A table's own
 * errors (full, reserved keys) are reported at its next synchronising call
 * (ht_sync, ht_size, ht_stats), as for ht_find_or_put.  HT_ERR_INVALID for a
 * NULL table, an item naming a table >= ntables, or n > 0 with NULL keys.
 * ------------------------------------------------------------------------- */
typedef struct ht_work {
    uint32_t table;          /* index into tables[] */
    uint32_t reserved_;
    const void* d_keys;
    uint64_t n;
    uint8_t* d_is_new;
} ht_work;

ht_status ht_multi_find_or_put(ht_table* const* tables, uint32_t ntables, const ht_work* h_list, uint32_t m,
                               void* stream);

/* ---------------------------------------------------------------------------
 * Batched exploration: `count` independent explorations (models of uneven
 * sizes) advanced together.  The paper times one kernel launch per batch
 * and table (Sections 4.1, 5); this form advances many tables' BFS levels
 * (Section 3.2) together.  Each exploration gets its own table of
 * h_capacity[i] slots (scheme h_schemes[i], bucket when h_schemes is NULL;
 * h_params: NULL or `count` parameter sets; key width 32 when the model's
 * vector fits 31 bits, else 64) and a states array holding its reachable
 * states in level order.  A step expands a share of every active
 * exploration's current level: advance the cursors and share the successor
 * buffer, generate successors, find-or-put them each against its own table
 * and append the new states.  Explorations are grouped by table kind (key
 * width, scheme, bucket shape).  Allocates everything at creation
 * (cudaMalloc), frees at destroy.  Errors: HT_ERR_INVALID (count 0 or
 * > 65536, a malformed model, a reserved initial state, max_levels 0 or
 * > 65536, a scheme other than HT_BUCKET / HT_CUCKOO), HT_ERR_OOM.
 * ------------------------------------------------------------------------- */
typedef struct ht_multi ht_multi;

ht_status ht_multi_create(uint32_t count, const ht_model* h_models, const uint64_t* h_s0,
                          const uint64_t* h_capacity, const ht_params* h_params, uint32_t max_levels,
                          void* stream, ht_multi** out);
ht_status ht_multi_create_ex(uint32_t count, const ht_model* h_models, const uint64_t* h_s0,
                             const uint64_t* h_capacity, const ht_scheme* h_schemes, const ht_params* h_params,
                             uint32_t max_levels, void* stream, ht_multi** out);

/* Empties every table and states array (required before every run but the
 * first after creation). */
ht_status ht_multi_reset(ht_multi* m, void* stream);

/* Runs every exploration to completion (or to max_levels / a full states
 * array).  mode 0: persistent -- one cooperative launch per group runs
 * every step of every exploration on the device, with grid-wide barriers
 * between the phases of a step; each barrier wait is bounded (2 s), and a
 * wait that runs out ends the launch and the call returns HT_ERR_TIMEOUT.
 * The host synchronises once, to read the results.  Bucket and Cuckoo
 * tables.  mode 1: the same steps as one launch per phase, the host reading
 * an activity flag after every step (bucket tables only); mode 2: one
 * exploration after another with ht_bfs (per-level launches for one table
 * at a time: the baseline; both schemes); mode 3: mode 1's step captured
 * once as a CUDA graph and replayed per step (bucket tables only).  Modes
 * 1 and 3 with a Cuckoo exploration: HT_ERR_INVALID.  max_steps 0 = no
 * limit beyond a safety bound.  HT_ERR_FULL when a table had to drop a key
 * (its capacity was too small for its exploration); the results are then
 * inexact.  Tables must be empty when a run starts (ht_multi_reset). */
ht_status ht_multi_run(ht_multi* m, int mode, uint64_t max_steps, void* stream);

/* Result of exploration i after a run: non-empty levels, states, successors
 * generated, complete flag, level sizes (host array of max_levels), the
 * device pointer of its states array (level order, key-width entries) and,
 * if h_states is non-NULL, a copy of up to h_states_cap of those states in
 * host memory (synchronises).  Every output pointer may be NULL. */
ht_status ht_multi_result(const ht_multi* m, uint32_t i, uint64_t* levels, uint64_t* states,
                          uint64_t* successors, int32_t* complete, uint64_t* h_level_sizes,
                          const void** d_states, void* h_states, uint64_t h_states_cap);

/* Steps the last run took (steps of the largest group in modes 0, 1 and 3;
 * the sum of the explorations' levels in mode 2). */
uint64_t ht_multi_steps(const ht_multi* m);

ht_status ht_multi_destroy(ht_multi* m);

/* Failure-detection test hooks of the persistent mode (mode 0), for tests
 * only.  barrier_timeout_ns: the bound on one grid-barrier wait (0 = the
 * default, 2 s).  absent_block: the index of one block of each persistent
 * launch that leaves before its first barrier, as a block that died would,
 * so that every other block's wait runs out (-1 = none, the default).  The
 * next ht_multi_run then returns HT_ERR_TIMEOUT within about the bound, the
 * device stays usable, and after ht_multi_reset (and the hooks set back to
 * 0, -1) runs are exact again.  HT_ERR_INVALID for NULL or absent_block <
 * -1.  Host only. */
ht_status ht_multi_test_hooks(ht_multi* m, uint64_t barrier_timeout_ns, int32_t absent_block);

/* ---------------------------------------------------------------------------
 * Serving: a request loop over many device-resident tables (64-bit keys).
 * A worker thread inside the library forms batches continuously: whenever
 * one of `max_inflight` batch slots is free it takes the oldest pending
 * request of every admitted table that has no request in flight, packs them
 * into one staging buffer and issues copy-in, one packed find-or-put launch
 * for all bucket-scheme tables of the batch (Cuckoo tables get their own
 * launches) and copy-out on the slot's stream.  A table's requests complete
 * in submission order, so each result equals what the request gets when the
 * requests of its table are run alone in that order.  Tables are admitted
 * when free device memory (cudaMemGetInfo, or fake_free_bytes for tests)
 * covers them plus hbm_reserve_bytes; requests for a table wait until it is
 * admitted.  The paper has no serving layer; it only states the problem
 * (Section 5: find-or-insert of a stream of elements).
 * ------------------------------------------------------------------------- */
typedef struct ht_server ht_server;

typedef struct ht_server_config {
    uint32_t max_inflight;            /* batch slots (streams), default 4, max 64 */
    uint32_t max_requests_per_batch;  /* default 4096, at most 2^20 */
    uint64_t batch_key_budget;        /* keys per batch, also the largest request; default 2^22 */
    uint64_t hbm_reserve_bytes;       /* device memory kept free, default 1 GiB */
    uint64_t fake_free_bytes;         /* tests: free memory to assume (0 = ask the driver) */
    int32_t pack;                     /* 1 (default): many tables per batch; 0: one request per batch */
    int32_t reserved_[3];
    ht_params table_params;           /* parameters of the bucket-scheme tables */
} ht_server_config;

typedef struct ht_server_stats {
    uint64_t requests;                /* completed since creation or the last reset */
    uint64_t keys;
    uint64_t batches;
    double seconds;                   /* wall time of the same period */
    double p50_us, p99_us, mean_us, max_us;   /* submit-to-result latency */
    uint64_t admitted_bytes;
    uint32_t tables_admitted;
    int32_t status;                   /* HT_OK, or the first error the worker met */
    /* Where the worker thread's time went over the same period: */
    double admit_seconds;             /* creating admitted tables (allocate + clear) */
    double pack_seconds;              /* packing requests into batches and issuing them */
    double finish_seconds;            /* copying results out of completed batches */
    double batch_us_mean;             /* mean issue-to-completion time of a batch (host view) */
    double batch_gpu_us_mean;         /* mean device time of a batch (events on its stream) */
    uint64_t tables_created;
    double inflight_seconds;          /* wall time with at least one batch in flight (host view) */
    uint64_t table_bytes_created;     /* device bytes of the tables created (each one cleared) */
} ht_server_stats;

ht_status ht_server_default_config(ht_server_config* cfg);
/* Starts the worker on the current device; allocates the batch slots. */
ht_status ht_server_create(const ht_server_config* cfg, ht_server** out);
/* Stops the worker (in-flight batches complete) and frees every table. */
ht_status ht_server_destroy(ht_server* s);
/* Registers a table of `capacity` slots; it is created once admitted. */
ht_status ht_server_open_table(ht_server* s, uint64_t capacity, ht_scheme scheme, uint32_t* table_id);
/* Frees the table after its pending requests complete. */
ht_status ht_server_close_table(ht_server* s, uint32_t table_id);
/* admitted: 1 admitted, 0 waiting, -1 closed; size: stored keys (0 while busy). */
ht_status ht_server_table_state(ht_server* s, uint32_t table_id, int32_t* admitted, uint64_t* size);
/* Queues a find-or-put of n keys (host memory, valid until the request
 * completes); h_is_new (nullable, n bytes, host) receives the flags.  Keys of
 * a large request (>= 2^16) in page-locked memory (cudaMallocHost,
 * cudaHostRegister) go to the device straight from h_keys; others are copied
 * through the server's own page-locked staging.
 * HT_ERR_INVALID if n exceeds batch_key_budget or the table is closing. */
ht_status ht_server_submit(ht_server* s, uint32_t table_id, const uint64_t* h_keys, uint64_t n,
                           uint8_t* h_is_new, uint64_t* request_id);
/* Waits up to timeout_ms for a request; HT_ERR_TIMEOUT if it is not done
 * (it stays queued and can be waited for again).  On completion returns the
 * request's status and forgets it. */
ht_status ht_server_wait(ht_server* s, uint64_t request_id, uint32_t timeout_ms, double* latency_us);
/* Counters and latency percentiles; reset != 0 starts a new period. */
ht_status ht_server_get_stats(ht_server* s, ht_server_stats* out, int reset);

/* ---------------------------------------------------------------------------
 * Kernel timing (CUDA events around every launch the library makes, on the
 * launch's stream).  ht_prof_read synchronises on the recorded events.
 * ------------------------------------------------------------------------- */
ht_status ht_prof_enable(int on);
ht_status ht_prof_reset(void);
/* Number of kernel kinds; names are stable strings. */
uint32_t ht_prof_num_kernels(void);
const char* ht_prof_kernel_name(uint32_t id);
ht_status ht_prof_read(uint32_t id, uint64_t* launches, double* total_ms);

/* ---------------------------------------------------------------------------
 * Random-access roofline probe (not part of the hash table): n_access reads
 * at uniformly random gran-aligned offsets of d_buf[0..bytes), folded into
 * *d_sink.  gran 8: one 8-byte load per access, eight in flight per thread
 * (a Cuckoo slot probe); gran 32: one 256-bit load per access, four in
 * flight per thread; gran 128: a 128-byte line read by 8 lanes with one
 * coalesced load (a bucket probe), four lines in flight per group.
 * ------------------------------------------------------------------------- */
ht_status ht_probe_random_read(const void* d_buf, uint64_t bytes, uint32_t gran,
                               uint64_t n_access, uint64_t seed,
                               unsigned long long* d_sink, void* stream);
/* The device address of the table's slot array and its size in bytes
 * (the words the scheme's kernels read and claim; 8 or 16 bytes per slot,
 * laid out as ht_create describes).  For tests and tools that inspect the
 * words or prepare a slot state on purpose; a caller that writes them must
 * keep the table's invariants.  Host only; HT_ERR_INVALID for NULL. */
ht_status ht_table_words(const ht_table* t, void** d_slots, uint64_t* bytes);

/* Random read-modify-write probe (not part of the hash table): n_access
 * 8-byte atomic adds of 1 at uniformly random 128-byte-aligned offsets of
 * d_buf[0..bytes) (the buffer's words change), eight in flight per thread;
 * each touches one line that L2 fetches from DRAM and later writes back, the
 * memory cost of a claim (CAS or exchange) in a random slot.  d_buf must be
 * 128-byte aligned and bytes >= 128, else HT_ERR_INVALID.  Asynchronous on
 * `stream`. */
ht_status ht_probe_random_rmw(void* d_buf, uint64_t bytes, uint64_t n_access, uint64_t seed, void* stream);

/* ---------------------------------------------------------------------------
 * Cuckoo find-or-put that allocates nothing.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- code
 * whose device memory is all reserved up front (an arena, or a framework's
 * caching allocator that already holds the GPU), or code on a path where an
 * allocation is not allowed (cudaMalloc can synchronise the device and is
 * refused during stream capture).  Such a caller supplies the table memory
 * itself; the per-call dedup set and winner list come from one static
 * device array inside the library (8 MiB, held on every GPU that uses the
 * library until the process exits).  No cudaMalloc or cudaFree is called.
 *
 * d_slots   caller-owned device array of nslots uint64 words: the table.
 * d_state   caller-owned device block of HT_NOALLOC_STATE_BYTES bytes,
 *           16-byte aligned: counters, a 101-word stash and a 64-word
 *           overflow area.  After the work completes:
 *             bytes 0..7    stored keys (uint64);
 *             bytes 8..15   keys dropped because no slot, stash or overflow
 *                           word was left (uint64; non-zero means the set is
 *                           incomplete: there is no rebuild);
 *             bytes 16..19  stash words in use (uint32);
 *             bytes 20..23  overflow words in use (uint32);
 *             bytes 24..27  sticky status bits (uint32): 1 = a reserved key
 *                           (top bit set) was seen and skipped, 2 = the
 *                           overflow area took a key (a regular table would
 *                           rebuild now), 4 = a key was dropped.
 *           The call itself returns HT_OK in all three cases: it does not
 *           synchronise, so these facts are only in the block.  Only a
 *           reset clears them.
 * seed      hash-constant seed; use the same seed for every call on a table.
 * d_keys    n uint64 keys, top bit 0; n <= HT_NOALLOC_MAX_BATCH, else
 *           HT_ERR_INVALID (split larger batches).
 * d_is_new  nullable; n bytes as in ht_find_or_put.
 * reset     non-zero: first empty the table and state (required on the
 *           first call for a table; uses fills, no allocation).
 * Semantics per call are those of ht_find_or_put on a Cuckoo table with 4
 * hash functions and an eviction bound of 256.
 * Every call looks up the static array's device address on the current
 * device (cudaGetSymbolAddress, a host-side lookup), so the address stays
 * right after a cudaDeviceReset; make the first call on a device before any
 * stream capture (it may load the library's module).
 * All calls share the array.  Each call with n > 0 first empties the whole
 * dedup set (a 4 MiB fill, a fixed cost of a few microseconds per call) and
 * zeroes its winner count, so no call depends on what an earlier, possibly
 * aborted, call left there.  Calls whose work overlaps on the GPU (other
 * streams, other host threads) race on the array: order them on one stream.
 * ------------------------------------------------------------------------- */
#define HT_NOALLOC_STATE_BYTES 2048
#define HT_NOALLOC_MAX_BATCH (1u << 18)
ht_status ht_cuckoo_find_or_put_noalloc(uint64_t* d_slots, uint64_t nslots, void* d_state,
                                        uint64_t seed, const uint64_t* d_keys, uint64_t n,
                                        uint8_t* d_is_new, int reset, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HT_H_ */
