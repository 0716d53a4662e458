/*
 * gconn.h -- C ABI of libgconn: static and incremental connected components
 * and spanning forests on one GPU (sm_103a), by concurrent union-find.
 *
 * The method is the two-phase framework of Hong, Dhulipala and Shun,
 * "Exploring the Design Space of Static and Incremental Graph Connectivity
 * Algorithms on GPUs" (PACT 2020): initialise labels, sample a subgraph,
 * find the most frequent label L_max, run a finish algorithm over the edges
 * of vertices whose label is not L_max, then finalise the labels
 * (Section 3.2, Algorithm 1); spanning forest (Algorithm 2); incremental
 * batches of inserts and queries (Section 3.5, Algorithm 3).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Vertex ids are uint32 in [0, n); n <= 0xFFFFFFFE (0xFFFFFFFF is reserved
 *   as "none").  Edge lists (COO) are interleaved uint32 pairs
 *   edges[2*i], edges[2*i+1].  CSR is offsets (uint64, n+1 entries,
 *   offsets[n] = number of arcs) plus cols (uint32); it must be symmetric
 *   (each undirected edge stored as both arcs) with every row sorted
 *   ascending, as in Section 2 ("Graph Notation and Formats").
 * - Self-loops and duplicate edges are accepted and change nothing.
 * - Edge, pair and query counts (m, b, q, count) are at most 2^60
 *   (E_INVAL above), so every byte size fits in 64 bits.
 * - Every pointer may be device memory or host memory (pageable or pinned);
 *   the library checks each one.  A host input that a call reads once or
 *   only in part (CSR columns; COO edges and insert / query batches for the
 *   union-find finishes) is read in place by the kernels when the device can
 *   address it: page-locked memory, or pageable memory on a device with
 *   coherent access to it (cudaDevAttrPageableMemoryAccess, e.g. over
 *   NVLink-C2C); other host inputs are copied to the device, as are all of
 *   them when the environment sets GCONN_HOST_STAGE=1.  Host inputs must not
 *   change while the call runs.  Host outputs are filled before the call
 *   returns.  The caller owns every buffer
 *   it passes; the library never frees caller memory.  Temporary device
 *   memory comes from the device's stream-ordered pool (cudaMallocAsync) and
 *   is returned on the same stream.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  With device-resident inputs and outputs every call only
 *   enqueues work and returns; errors found on the device (an endpoint >= n,
 *   an iteration cap reached) are reported by the next gconn_sync() on that
 *   device.  With any host output the call synchronises the stream and
 *   returns the device status itself.  Device error flags are per device and
 *   shared by all calls on it.
 * - Results are the canonical labelling: labels[v] = the smallest vertex id
 *   of v's component, whatever variant computed them.
 */
#ifndef GCONN_H
#define GCONN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
typedef enum gconn_status {
    GCONN_OK = 0,
    GCONN_E_INVAL = 1,          /* null pointer, bad size or malformed argument */
    GCONN_E_RANGE = 2,          /* an endpoint or query vertex is >= n */
    GCONN_E_NOMEM = 3,          /* device allocation failed */
    GCONN_E_UNSUPPORTED = 4,    /* invalid variant combination for this input */
    GCONN_E_NONCONVERGED = 5,   /* a device loop reached its iteration cap */
    GCONN_E_CUDA = 6            /* a CUDA runtime call failed */
} gconn_status;

/* --------------------------------------------------------------- variants */
/* Sampling phase (Section 3.3; Algorithms 2-4 of the appendix).  Sampling
 * needs CSR input: the skip rule drops whole adjacency lists. */
enum { GCONN_SAMPLE_NONE = 0, GCONN_SAMPLE_KOUT = 1, GCONN_SAMPLE_HB = 2, GCONN_SAMPLE_BFS = 3 };

/* Finish algorithm (Section 3.4): union-find rules (Algorithms 7-11 and
 * Union-JTB), the finish rules of ECL-CC (Union-Async with path splitting)
 * and Afforest, root-based Shiloach-Vishkin (Algorithm 12), Liu-Tarjan,
 * Label Propagation and Stergiou's algorithm.  LP and Stergiou are not
 * root-based: components only (no forest, no incremental handle). */
enum {
    GCONN_LINK_ASYNC = 0, GCONN_LINK_HOOKS = 1, GCONN_LINK_EARLY = 2,
    GCONN_LINK_REMCAS = 3, GCONN_LINK_JTB = 4, GCONN_LINK_SV = 5, GCONN_LINK_LT = 6,
    GCONN_LINK_REMLOCK = 7, GCONN_LINK_ECLCC = 8, GCONN_LINK_AFFOREST = 9,
    GCONN_LINK_LP = 10, GCONN_LINK_STERGIOU = 11
};

/* On-the-fly compression (Algorithm 5).  FULLSHORTCUT = no on-the-fly
 * compression; the separate pointer-jumping pass (run after sampling and at
 * finalisation for every variant) does all of it.  TWOTRYSPLIT is Union-JTB
 * only; COMPRESS is not valid with Union-Rem-CAS (Section 3.4). */
enum {
    GCONN_FIND_NAIVE = 0, GCONN_FIND_COMPRESS = 1, GCONN_FIND_SPLIT = 2,
    GCONN_FIND_HALVE = 3, GCONN_FIND_TWOTRYSPLIT = 4, GCONN_FIND_FULLSHORTCUT = 5
};

/* Splice step of Rem's algorithms (Algorithm 6); NONE selects SPLICE. */
enum { GCONN_SPLICE_NONE = 0, GCONN_SPLICE_SPLIT_ONE = 1, GCONN_SPLICE_HALVE_ONE = 2, GCONN_SPLICE_SPLICE = 3 };

/* Liu-Tarjan rule set (appendix list of 16 variants): connect rule in the
 * low two bits, then flags.  E.g. PRS = GCONN_LT_PARENT | GCONN_LT_ROOTUPDATE. */
enum {
    GCONN_LT_CONNECT = 0, GCONN_LT_PARENT = 1, GCONN_LT_EXTENDED = 2,
    GCONN_LT_ROOTUPDATE = 4, GCONN_LT_FULLSHORTCUT = 8, GCONN_LT_ALTER = 16
};

typedef struct gconn_variant {
    int32_t sample;     /* GCONN_SAMPLE_* */
    int32_t k;          /* k-out: edges per vertex (first k; default 2) */
    int32_t hb_n;       /* HB: edges per remaining root (default 4) */
    int32_t link;       /* GCONN_LINK_* */
    int32_t find;       /* GCONN_FIND_* */
    int32_t splice;     /* GCONN_SPLICE_* (Union-Rem-CAS / Union-Rem-Lock only) */
    int32_t lt_rules;   /* GCONN_LT_* bits (Liu-Tarjan only) */
    int32_t block;      /* threads per block of the finish kernels, 0 = library default (256);
                           a multiple of 32 in [64, 1024], values above 256 run as 256 */
    uint64_t seed;      /* L_max / BFS-source sampling and Union-JTB priorities */
    uint32_t iter_cap;  /* per-operation loop cap, 0 = default (2^24) */
    uint32_t ablation;  /* 0 = the library's kernels; GCONN_ABL_* bits select plain forms
                           for measurement (results are the same) */
} gconn_variant;

/* Ablation bits (measurement only, CSR input; no paper counterpart beyond the
 * optimisations they switch off, Section 3.3):
 *   GCONN_ABL_PLAIN_SAMPLE: k-out sampling with one thread per vertex walking
 *     its first k arcs (no per-warp packing of unions, no deferral);
 *   GCONN_ABL_NO_VG: no vertex gathering -- full compression, then a finish
 *     with one thread per vertex over its whole row, skipping vertices whose
 *     parent is L_max (no active lists, no load balancing). */
#define GCONN_ABL_PLAIN_SAMPLE 1u
#define GCONN_ABL_NO_VG 2u

/* Fill *v with the library default: Union-Rem-CAS with naive find and
 * SplitAtomicOne (the fastest finish measured on GB300 on RMAT scale 22, with
 * and without sampling; Section 4 finds Union-Async and Union-Rem-CAS the
 * fastest rules), k-out k=2 sampling for CSR input and no sampling for COO
 * input.  Returns GCONN_E_INVAL on NULL. */
gconn_status gconn_variant_default(gconn_variant* v);

/* Validate a variant for an input kind (0 = COO, 1 = CSR) and a purpose
 * (0 = components, 1 = spanning forest, 2 = incremental handle).  Returns
 * GCONN_OK, GCONN_E_INVAL (value out of range) or GCONN_E_UNSUPPORTED (e.g.
 * sampling on COO, COMPRESS with Rem-CAS, splice without Rem-CAS, TWOTRYSPLIT
 * without JTB; for forests and incremental handles a Liu-Tarjan rule set
 * without RootUpdate; for forests Rem-CAS with SpliceAtomic, which moves
 * non-roots between trees and so is not root-based in the sense of
 * Section 2). */
gconn_status gconn_variant_check(const gconn_variant* v, int input_kind, int purpose);

/* -------------------------------------------------------- static: COO */
/* Connected components of the graph with n vertices and m undirected edges
 * (Algorithm 1 without a sampling phase; COO input, Section 2).
 *   edges  : uint32[2m] interleaved pairs (device or host)
 *   labels : uint32[n] output, canonical min-id labels (device or host)
 *   v      : variant or NULL for the default; sampling must be NONE.
 * labels doubles as the union-find parent array while the call runs.
 * Errors: E_INVAL (null pointer with n or m > 0, n = 0xFFFFFFFF, unknown ablation bits),
 * E_UNSUPPORTED (see gconn_variant_check), E_RANGE (endpoint >= n),
 * E_NONCONVERGED, E_NOMEM, E_CUDA. */
gconn_status gconn_cc(uint32_t n, uint64_t m, const uint32_t* edges, uint32_t* labels,
                      const gconn_variant* v, void* stream);

/* -------------------------------------------------------- static: CSR */
/* Connected components from symmetric sorted CSR with the full two-phase
 * method (Algorithm 1): sampling (k-out, HB or BFS), L_max, finish over the
 * adjacency of vertices whose sampled label is not L_max, finalisation.
 *   offsets : uint64[n+1], cols : uint32[offsets[n]]
 *   labels  : uint32[n] output, canonical min-id labels.
 * Errors as gconn_cc. */
gconn_status gconn_cc_csr(uint32_t n, const uint64_t* offsets, const uint32_t* cols,
                          uint32_t* labels, const gconn_variant* v, void* stream);

/* The same with uint32 offsets, for graphs with fewer than 2^32 arcs
 * (Section 2's CSR with 4-byte row offsets): identical labels, half the
 * offset bytes read by the sampling and gathering kernels.
 *   offsets : uint32[n+1] (4-byte aligned), cols : uint32[offsets[n]]
 * Errors as gconn_cc_csr. */
gconn_status gconn_cc_csr32(uint32_t n, const uint32_t* offsets, const uint32_t* cols,
                            uint32_t* labels, const gconn_variant* v, void* stream);

/* ---------------------------------------------- sampling instrumentation */
/* The quantities of Section 4.3 (Table 4 and the edges-inspected figure) for
 * one CSR run: after the sampling phase, Cov = lmax_vertices / n (vertices in
 * the L_max component, whose arcs the finish skips), IC =
 * inter_component_arcs / arcs (arcs whose endpoints have different sampled
 * labels), Time % = sample_ms / total_ms, plus the arcs the sampling step
 * inspected (k-out, HB; 0 for BFS and none) and the finish's active vertices
 * and arcs.  The run is a separate counting pass (extra kernels, one host
 * synchronisation), not the timed path.  Device buffers only; labels receives
 * the canonical labels.  Union-JTB and the round-based finishes:
 * GCONN_E_UNSUPPORTED. */
typedef struct gconn_sample_stats {
    uint64_t n, arcs;
    uint64_t lmax_vertices;          /* Cov numerator */
    uint64_t sampled_components;     /* roots after sampling */
    uint64_t active_vertices;        /* label != L_max and degree > 0 */
    uint64_t active_arcs;            /* arcs of the active vertices */
    uint64_t inter_component_arcs;   /* IC numerator */
    uint64_t sample_arcs_inspected;
    uint64_t lmax;                   /* the chosen L_max (0xFFFFFFFF without sampling) */
    double sample_ms, total_ms;      /* CUDA events: init through sampling, L_max and gathering;
                                        the whole pass without the counting kernel */
} gconn_sample_stats;
gconn_status gconn_cc_csr_stats(uint32_t n, const uint64_t* offsets, const uint32_t* cols, uint32_t* labels,
                                const gconn_variant* v, gconn_sample_stats* out, void* stream);

/* ------------------------------------------------------ spanning forest */
/* Spanning forest (Algorithm 2): every root that stops being a root records
 * the input edge that linked it (Section 3.2).  Output ids are COO edge
 * indices in [0, m), written unsorted to forest[0 .. count-1] (capacity n);
 * count = n - (number of components).  m must be < 2^32 - 1.
 *   forest       : uint64[n] output (device or host)
 *   forest_count : uint64[1] output (device or host)
 *   labels       : optional uint32[n] canonical labels (NULL = not wanted)
 * Variant: no sampling; Liu-Tarjan only with RootUpdate rule sets; Rem-CAS
 * only with SplitAtomicOne or HalveAtomicOne. */
gconn_status gconn_spanning_forest(uint32_t n, uint64_t m, const uint32_t* edges,
                                   uint64_t* forest, uint64_t* forest_count, uint32_t* labels,
                                   const gconn_variant* v, void* stream);

/* Spanning forest from symmetric sorted CSR with sampling.  Output ids are
 * arc positions a in [0, offsets[n]); arc a joins the row containing a to
 * cols[a].  offsets[n] must be < 2^32 - 1.  Otherwise as above. */
gconn_status gconn_spanning_forest_csr(uint32_t n, const uint64_t* offsets, const uint32_t* cols,
                                       uint64_t* forest, uint64_t* forest_count, uint32_t* labels,
                                       const gconn_variant* v, void* stream);
/* The same with uint32 offsets (offsets[n] < 2^32 - 1). */
gconn_status gconn_spanning_forest_csr32(uint32_t n, const uint32_t* offsets, const uint32_t* cols,
                                         uint64_t* forest, uint64_t* forest_count, uint32_t* labels,
                                         const gconn_variant* v, void* stream);

/* ---------------------------------------------------------- incremental */
/* Incremental connectivity (Section 3.5, Algorithm 3).  The handle owns a
 * device-resident union-find over n vertices, initialised to singletons (an
 * empty initial graph; insert a batch to start from a non-empty one).  Only
 * root-based finish algorithms are allowed: the union-find rules, SV, and the
 * Liu-Tarjan rule sets with RootUpdate; sampling must be NONE.
 * Semantics (phase-concurrent, which Rem-CAS with splicing needs): a query
 * batch sees exactly the union of all insert batches submitted before it on
 * the handle; insert batches commute.  Calls on one handle must be ordered
 * (same stream, or synchronised); the handle is not thread-safe.
 * gconn_inc_create: *out receives the handle.  Errors: E_INVAL, E_UNSUPPORTED,
 * E_NOMEM, E_CUDA. */
typedef struct gconn_inc gconn_inc;
gconn_status gconn_inc_create(uint32_t n, const gconn_variant* v, void* stream, gconn_inc** out);

/* Insert b undirected edges (uint32[2b] pairs, device or host).  E_RANGE is
 * reported through gconn_sync (or directly when the input is on the host). */
gconn_status gconn_inc_insert_batch(gconn_inc* h, uint64_t b, const uint32_t* edges, void* stream);

/* Answer q connectivity queries (Section 2): connected[i] = 1 iff pairs[2i]
 * and pairs[2i+1] are in one component given every insert submitted before.
 * pairs: uint32[2q]; connected: uint8[q] (device or host). */
gconn_status gconn_inc_query(gconn_inc* h, uint64_t q, const uint32_t* pairs, uint8_t* connected,
                             void* stream);

/* A mixed batch as in Algorithm 3: op i is a query when is_query[i] != 0,
 * else an insert.  Bit i of result_bits (uint32 words, ceil(b/32) of them,
 * bit i%32 of word i/32) is 1 iff op i is a query whose endpoints are
 * connected.  Inserts and queries of the batch run concurrently, so an answer
 * is linearizable: 1 whenever the endpoints were connected before the batch,
 * 0 whenever they are not connected after it, either in between.  For
 * Union-Rem-CAS / Rem-Lock the batch's inserts run first, then its queries
 * (Section 3.5).  Round-based finishes: GCONN_E_UNSUPPORTED.
 *   pairs: uint32[2b]; is_query: uint8[b]; result_bits: uint32[ceil(b/32)]. */
gconn_status gconn_inc_process_batch(gconn_inc* h, uint64_t b, const uint32_t* pairs, const uint8_t* is_query,
                                     uint32_t* result_bits, void* stream);

/* Edge inspections of the handle's insert work, the quantity of Section 4.4's
 * edges-inspected figure (Shiloach-Vishkin and Liu-Tarjan per batch size):
 * a union-find finish reads each edge of an insert batch once (b per batch,
 * and b per mixed batch of b ops); the round-based finishes re-read the whole
 * batch every round until the labels converge (rounds x b, counted on the
 * host, which already waits for each round's convergence flag).
 *   *last_batch : inspections of the most recent insert or mixed batch
 *   *total      : since the handle was created
 * Queries are not counted.  Errors: E_INVAL on a NULL argument. */
gconn_status gconn_inc_edges_inspected(const gconn_inc* h, uint64_t* last_batch, uint64_t* total);

/* Canonical min-id labels of the current state into uint32[n] (device or host). */
gconn_status gconn_inc_labels(gconn_inc* h, uint32_t* labels, void* stream);

/* Release the handle and its device memory (synchronises its last stream). */
gconn_status gconn_inc_destroy(gconn_inc* h);

/* --------------------------------------------------------------- serving */
/* No paper counterpart for the loop itself; each request is an incremental
 * insert or query batch (Section 3.5).  A server owns sessions (one
 * device-resident union-find each, as gconn_inc) and a worker thread that
 * admits submitted requests while device memory (cfg.device_budget_bytes of
 * staging) and stream slots (cfg.slots) are free, coalesces consecutive
 * requests of one session and kind (up to cfg.coalesce_pairs pairs) into one
 * launch, and runs different sessions' launches concurrently.  Per session a
 * query sees exactly the inserts submitted before it: a run of inserts, or of
 * queries, starts only after the session's previous run finished.
 * Requests use host (or device) buffers, which must stay valid until
 * gconn_server_wait returns for that ticket; answers are written to `result`
 * (uint8 per pair).  Where the device can use a request's buffers in place
 * (device memory; page-locked host memory; pageable host memory on a device
 * with coherent access to it) the kernels read the pairs and write the
 * answers there directly; otherwise they are staged through pinned buffers of
 * cfg.slot_pairs pairs.  A merged launch holds at most cfg.slot_pairs pairs:
 * a larger request runs alone (a small request merged with it would wait for
 * it).
 * gconn_server_wait blocks until the request completed and gives its latency
 * (submit to answer available, host clock); each ticket is waited for once
 * (a second wait, or a ticket never issued, returns E_INVAL).  All calls are
 * thread-safe. */
enum { GCONN_OP_INSERT = 0, GCONN_OP_QUERY = 1 };
typedef struct gconn_server_config {
    uint64_t device_budget_bytes;  /* staging bytes allowed in flight (default 4 GiB) */
    uint32_t slots;                /* concurrent launches / streams (default 8) */
    uint32_t coalesce_pairs;       /* max pairs merged into one launch (default 2^22) */
    uint32_t slot_pairs;           /* pinned staging per slot, in pairs (default 2^22) */
    uint32_t reserved;
} gconn_server_config;
typedef struct gconn_server gconn_server;
gconn_status gconn_server_config_default(gconn_server_config* c);
gconn_status gconn_server_create(const gconn_server_config* cfg, gconn_server** out);
gconn_status gconn_server_open_session(gconn_server* s, uint32_t n, const gconn_variant* v, uint32_t* session);
gconn_status gconn_server_submit(gconn_server* s, uint32_t session, int op, uint64_t count,
                                 const uint32_t* pairs, uint8_t* result, uint64_t* ticket);
gconn_status gconn_server_wait(gconn_server* s, uint64_t ticket, double* latency_ms);
/* Canonical labels of a session after every request submitted so far (host buffer). */
gconn_status gconn_server_labels(gconn_server* s, uint32_t session, uint32_t* labels);
gconn_status gconn_server_close_session(gconn_server* s, uint32_t session);
gconn_status gconn_server_stats(gconn_server* s, uint64_t* launches, uint64_t* groups, uint64_t* requests);
/* Finishes every submitted request, then releases everything. */
gconn_status gconn_server_destroy(gconn_server* s);

/* ----------------------------------------------------- captured plans */
/* No paper counterpart.  The whole static pass for one input (the same work
 * as gconn_cc / gconn_cc_csr on the same arguments) captured once into a CUDA
 * graph; gconn_plan_run replays it on `stream`, so a repeated computation on
 * the same buffers (their contents may change between runs) costs one graph
 * launch instead of one host launch per kernel.  All buffers must be device
 * memory and stay alive while the plan exists.  Variants whose pass reads a
 * device flag on the host every round (BFS sampling, SV, Liu-Tarjan) cannot
 * be captured: GCONN_E_UNSUPPORTED.  Device-side errors come back from
 * gconn_sync.  If profiling is on while a plan is created, its kernels' event
 * pairs are captured too and each replay queues them for gconn_profile_sync. */
typedef struct gconn_plan gconn_plan;
gconn_status gconn_plan_create_cc(uint32_t n, uint64_t m, const uint32_t* edges, uint32_t* labels,
                                  const gconn_variant* v, gconn_plan** out);
gconn_status gconn_plan_create_cc_csr(uint32_t n, const uint64_t* offsets, const uint32_t* cols,
                                      uint32_t* labels, const gconn_variant* v, gconn_plan** out);
/* The spanning-forest pass of gconn_spanning_forest_csr (Algorithm 2) as a
 * plan: forest, forest_count and (optional) labels must be device memory. */
gconn_status gconn_plan_create_forest_csr(uint32_t n, const uint64_t* offsets, const uint32_t* cols,
                                          uint64_t* forest, uint64_t* forest_count, uint32_t* labels,
                                          const gconn_variant* v, gconn_plan** out);
/* The plans of gconn_cc_csr32 and gconn_spanning_forest_csr32 (uint32 offsets). */
gconn_status gconn_plan_create_cc_csr32(uint32_t n, const uint32_t* offsets, const uint32_t* cols,
                                        uint32_t* labels, const gconn_variant* v, gconn_plan** out);
gconn_status gconn_plan_create_forest_csr32(uint32_t n, const uint32_t* offsets, const uint32_t* cols,
                                            uint64_t* forest, uint64_t* forest_count, uint32_t* labels,
                                            const gconn_variant* v, gconn_plan** out);
gconn_status gconn_plan_run(gconn_plan* p, void* stream);
gconn_status gconn_plan_destroy(gconn_plan* p);

/* ------------------------------------------------------ batched graphs */
/* Connected components of G independent graphs in one go (no paper
 * counterpart for the batching itself; each graph gets Algorithm 1 without
 * sampling on COO input).  Graph g has vertices [vtx_off[g], vtx_off[g+1])
 * and edges [edge_off[g], edge_off[g+1]) of the concatenated arrays; its
 * edges use LOCAL ids in [0, n_g) and its labels are LOCAL min ids.
 * Graphs with n_g <= class_max_n[last] run entirely in shared memory (32-bit
 * parents up to n_g = 58,112, 16-bit above, one CTA per graph, one persistent kernel per size class on its own
 * stream); larger graphs use the global-memory path one launch each.
 *   vtx_off, edge_off : uint64[G+1] (device or host; read on the host once)
 *   edges             : uint32[2 * edge_off[G]] pairs, DEVICE memory
 *   labels            : uint32[vtx_off[G]] output, DEVICE memory
 * The tune table picks block size and union rule per size class; NULL = the
 * default table, gconn_batch_autotune measures one. */
#define GCONN_BATCH_CLASSES 4
typedef struct gconn_batch_tune {
    uint32_t class_max_n[GCONN_BATCH_CLASSES]; /* inclusive upper n of each class, ascending, <= 65536 */
    int32_t block[GCONN_BATCH_CLASSES];        /* threads per CTA (multiple of 32, <= 1024) */
    int32_t link[GCONN_BATCH_CLASSES];         /* GCONN_LINK_ASYNC or GCONN_LINK_REMCAS */
    int32_t find[GCONN_BATCH_CLASSES];         /* GCONN_FIND_NAIVE or GCONN_FIND_HALVE (Async only) */
} gconn_batch_tune;

gconn_status gconn_batch_tune_default(gconn_batch_tune* t);

/* One-shot: plan, run and wait.  Errors: E_INVAL (offsets not monotone, a
 * graph with more than 0xFFFFFFFE vertices, more than 2^60 edges in all, host
 * edges / labels, misaligned edges, bad tune table), E_UNSUPPORTED, E_NOMEM,
 * E_CUDA; E_RANGE (local endpoint >= n_g) via gconn_sync. */
gconn_status gconn_cc_batched(uint32_t G, const uint64_t* vtx_off, const uint64_t* edge_off,
                              const uint32_t* edges, uint32_t* labels, const gconn_batch_tune* tune,
                              void* stream);

/* Reusable plan bound to the given device buffers: the size classes, the
 * largest-first order and the whole launch sequence captured once into a CUDA
 * graph.  gconn_batch_run replays it on `stream` (asynchronous; the buffers
 * must stay alive and may be refilled between runs); destroy frees the plan
 * (after a device synchronisation). */
typedef struct gconn_batch gconn_batch;
gconn_status gconn_batch_create(uint32_t G, const uint64_t* vtx_off, const uint64_t* edge_off,
                                const uint32_t* edges, uint32_t* labels, const gconn_batch_tune* tune,
                                void* stream, gconn_batch** out);
gconn_status gconn_batch_run(gconn_batch* b, void* stream);
gconn_status gconn_batch_destroy(gconn_batch* b);

/* Measure a tune table for this batch: every (block in {128,256,512,1024},
 * rule in {Async+naive, Async+halving, Rem-CAS+SplitAtomicOne}) on each size
 * class alone, median of three timed runs, best kept in *out.  Writes labels
 * as a side effect.  Synchronous. */
gconn_status gconn_batch_autotune(uint32_t G, const uint64_t* vtx_off, const uint64_t* edge_off,
                                  const uint32_t* edges, uint32_t* labels, gconn_batch_tune* out,
                                  void* stream);

/* ------------------------------------------- components without allocation */
/* No counterpart in the paper: this call exists for callers that must not
 * allocate device memory -- for example when another allocator (a
 * framework's caching pool) already owns the GPU's memory, or when a serving
 * process runs under a fixed memory budget in which a new allocation could
 * fail or stall the device.  It computes the same canonical labels as
 * gconn_cc_csr, for the same inputs, without any device allocation.
 *   n                 : at most GCONN_NOALLOC_MAX_N, else GCONN_E_INVAL
 *   offsets, cols     : device memory only (no host staging), as gconn_cc_csr
 *   labels            : device memory only, uint32[n] output
 *   v                 : sampling NONE, KOUT or HB; link ASYNC, EARLY or
 *                       REMCAS (others give GCONN_E_UNSUPPORTED)
 * Its scratch (about 16.2 MiB) is one fixed device array inside libgconn.
 * All calls share that array and it keeps the previous call's contents, so
 * calls whose GPU work overlaps (other streams, other threads) race:
 * serialise them.  The first call on each device sets up: it looks the array
 * up (cudaGetSymbolAddress) and loads the code of every kernel this call can
 * launch.  Under lazy module loading (the CUDA default) that set-up is when
 * the driver maps the array and the code, so it is the one call that takes
 * device memory; from then on the GPU holds them until the process exits.  A
 * call with n == 0 does the set-up and nothing else (its pointers are not
 * read): make it on each device before handing the memory to another
 * allocator, and before any stream capture.  Like gconn_cc_csr with device
 * buffers, it only enqueues work: device-side errors come back from
 * gconn_sync. */
#define GCONN_NOALLOC_MAX_N 1048576u
gconn_status gconn_cc_csr_noalloc(uint32_t n, const uint64_t* offsets, const uint32_t* cols,
                                  uint32_t* labels, const gconn_variant* v, void* stream);

/* ------------------------------------------------------------ utilities */
/* Wait for `stream`, then return and clear the device error flags of the
 * current device (GCONN_E_RANGE, GCONN_E_NONCONVERGED) or GCONN_E_CUDA. */
gconn_status gconn_sync(void* stream);

/* Static description of a status code. */
const char* gconn_status_str(gconn_status s);

/* Kernel launches made by this library in this process (all devices). */
uint64_t gconn_launch_count(void);

/* Memory utility; the paper has no counterpart.  Scratch and host-input
 * staging buffers are taken from one stream-ordered memory pool per device
 * that keeps freed memory reserved for later calls (so repeated calls do not
 * map and unmap device memory).  gconn_release_cached returns the pool's idle
 * memory on the current device to the system.  Memory whose stream-ordered
 * free has not executed yet stays reserved: synchronise the streams used
 * first.  Returns GCONN_OK or GCONN_E_CUDA. */
gconn_status gconn_release_cached(void);

/* Per-kernel timing with CUDA events recorded on each launch's own stream.
 * gconn_profile_enable(1) starts recording (0 stops), gconn_profile_reset
 * clears the totals, gconn_profile_get(i, ...) synchronises pending events and
 * returns the name, launch count and summed milliseconds of the i-th kernel
 * (GCONN_E_INVAL once i is past the last one). */
gconn_status gconn_profile_enable(int on);
/* Restricts the timing to the kernels named in a comma-separated list (the
 * names gconn_profile_get reports, e.g. "kout,vg"); NULL or "" times every
 * kernel again.  Applies to launches and plan captures made afterwards.  Each
 * timed kernel adds two event records to a captured plan, and each record
 * serialises the replay for a few microseconds, so timing one kernel disturbs
 * a pass far less than timing all of them. */
gconn_status gconn_profile_select(const char* names);
gconn_status gconn_profile_reset(void);
/* Collect every queued event pair now (waits for them).  Needed after each
 * replay of a profiled plan, whose events re-record on every replay. */
gconn_status gconn_profile_sync(void);
gconn_status gconn_profile_get(int i, const char** name, uint64_t* launches, double* total_ms);

#ifdef __cplusplus
}
#endif
#endif /* GCONN_H */
