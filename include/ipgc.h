/*
 * ipgc.h -- C ABI of libipgc.so: hybrid IPGC graph colouring on one GB300.
 *
 * The library colours an undirected graph with the Iterative Parallel Graph
 * Coloring (IPGC) loop of "A Hybrid Graph Coloring Algorithm for GPUs"
 * (Section II-C): every uncoloured node takes the smallest colour not used by
 * its neighbours (first fit, the footnote's mex), conflicting endpoints are
 * uncoloured again, and the loop repeats until the worklist of uncoloured
 * nodes is empty. Each iteration runs either topology-driven (sweep every
 * node) or data-driven (sweep the worklist), chosen from the worklist size
 * (Section IV, threshold H, about 60 % of the node count); the worklist is
 * kept up to date in every iteration, in both modes (Sections I and IV).
 *
 * Result semantics (fixed, deterministic; the same for every mode, driver and
 * entry point):
 *   - colour 0 means "uncoloured"; valid colours are 1, 2, ...;
 *   - tentative colours are taken from the snapshot of committed colours at
 *     the start of the round (active neighbours count as uncoloured);
 *   - of two adjacent active nodes with the same tentative colour the one
 *     with the higher node ID loses and stays in the worklist;
 *   - one round = one assignment step + one conflict step; the last,
 *     conflict-free round is counted; num_colors = the largest colour.
 *
 * Graph input: CSR with int32 rowptr[n + 1] and int32 col[nnz] (directed
 * entries, both directions of every undirected edge), no self-loops, no
 * duplicate entries, every row sorted ascending (the paper removes self
 * loops and multi-edges before colouring, Section V). nnz < 2^31.
 *
 * Conventions for every entry point:
 *   - returns IPGC_OK (0), IPGC_PENDING (1) or a negative IPGC_ERR_* code;
 *     never aborts, never prints, never throws across the ABI;
 *   - "device pointer" arguments are CUDA device memory on the context's
 *     device, owned by the caller, which must stay valid until the call has
 *     completed on its stream; "host pointer" arguments are plain host memory;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream);
 *   - the library allocates only its own workspace, held in the context and
 *     released by ipgc_ctx_destroy.
 */
#ifndef IPGC_H
#define IPGC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define IPGC_API __attribute__((visibility("default")))
#else
#define IPGC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define IPGC_OK 0
#define IPGC_PENDING 1
#define IPGC_ERR_INVALID (-1)     /* bad argument or CSR (see ipgc_validate_csr) */
#define IPGC_ERR_OOM (-2)         /* device or host allocation failed */
#define IPGC_ERR_TIMEOUT (-3)     /* a bounded device-side wait expired */
#define IPGC_ERR_NO_CONVERGE (-4) /* more than max_rounds rounds */
#define IPGC_ERR_CUDA (-5)        /* a CUDA call failed; see ipgc_ctx_cuda_error */
#define IPGC_ERR_BUSY (-6)        /* server: request not admissible right now */
#define IPGC_ERR_UNSUPPORTED (-7) /* option combination not available */
#define IPGC_ERR_NOT_FOUND (-8)   /* server: unknown ticket */
#define IPGC_ERR_TOO_LARGE (-9)   /* graph above a fixed-size entry point's limits */

/* Mode policy: how each round chooses topology- or data-driven work. */
#define IPGC_MODE_THRESHOLD 0 /* topology iff |WL| > floor(threshold_frac * n) (Section IV) */
#define IPGC_MODE_TOPO 1      /* every round topology-driven (still pushes the worklist) */
#define IPGC_MODE_DATA 2      /* every round data-driven ("Plain" IPGC, Section II-C) */
#define IPGC_MODE_LEARNED 3   /* per-round MLP loaded by ipgc_policy_load; threshold fallback */

/* Driver: where the round loop runs (the paper's Iteration Outlining, Section V). */
#define IPGC_DRIVER_PERSISTENT 0 /* one cooperative launch, rounds separated by grid barriers */
#define IPGC_DRIVER_HOSTLOOP 1   /* one launch per phase, host reads |WL| after every round */

typedef struct ipgc_ctx ipgc_ctx;

typedef struct ipgc_stats {
  int32_t rounds;          /* rounds executed */
  int32_t num_colors;      /* largest colour = number of distinct colours */
  int32_t rounds_topo;     /* rounds run topology-driven */
  int32_t rounds_data;     /* rounds run data-driven */
  int64_t edges_processed; /* sum over rounds of the degrees of the active nodes */
  uint64_t ns;             /* device time of the colouring loop (%globaltimer) */
  int32_t error;           /* IPGC_OK or the error the device reported */
  int32_t filter_round;    /* first round with neighbour filtering (0: none; see
                              ipgc_options.filter_degree); always 0 for batches */
} ipgc_stats;

/* One record per round, written to ipgc_options.trace when it is non-NULL. */
typedef struct ipgc_trace_rec {
  int32_t round;      /* 1-based */
  int32_t mode;       /* IPGC_MODE_TOPO or IPGC_MODE_DATA: how this round ran */
  int64_t wl_size;    /* |WL| at the start of the round */
  int64_t deg_sum;    /* sum of deg(v) over the worklist */
  int32_t max_color;  /* largest committed colour at the start of the round */
  int32_t shortcut;   /* 1 for round 1, whose assignment step is implicit */
  int32_t wl_small;   /* worklist nodes of degree <= t1 */
  int32_t push_ns;    /* IPGC_FORBIDDEN_PUSH: ns of the push phase after the conflict step
                         (included in t_detect); 0 otherwise */
  uint64_t t_begin;   /* %globaltimer at the start of the round (ns) */
  uint64_t t_assign;  /* ... after the assignment step's grid barrier */
  uint64_t t_detect;  /* ... after the conflict step's grid barrier */
} ipgc_trace_rec;

typedef struct ipgc_options {
  int32_t mode;           /* IPGC_MODE_*; default THRESHOLD */
  float threshold_frac;   /* H = floor(threshold_frac * n); default 0.6 (Section IV) */
  int32_t driver;         /* IPGC_DRIVER_*; default PERSISTENT */
  int32_t max_rounds;     /* 0 = n + 1, which always suffices */
  uint64_t timeout_ns;    /* limit for each device-side wait; 0 = 10 s */
  int32_t validate;       /* 1 = check the CSR on the device first (IPGC_ERR_INVALID) */
  int32_t t1;             /* degree <= t1 (<= 255): a warp colours 32 such nodes together;
                             0 = chosen on the device: the largest degree when it is <= 255
                             (every node on the low-degree path), else 64 */
  int32_t chunk;          /* degree > t1: the node's neighbours are cut into work items of
                             this many (32..4096), one warp each; 0 = default 1024 */
  int32_t block_size;     /* threads per CTA of the colouring kernel; 0 = default */
  int32_t blocks_per_sm;  /* resident CTAs per SM; 0 = as many as fit */
  ipgc_trace_rec* trace;  /* device pointer to trace_cap records, or NULL */
  int32_t* fin_round;     /* device pointer to int32[n] receiving the round in which each
                             node's colour was committed, or NULL */
  int32_t trace_cap;
  int32_t fault_inject;   /* tests only: 1 = every grid barrier also waits for a CTA that
                             never arrives, so the launch ends with IPGC_ERR_TIMEOUT after
                             timeout_ns (exercises the bounded waits); 0 otherwise */
  float policy_margin;    /* IPGC_MODE_LEARNED: when the network's probability p of "topology
                             is faster" has |p - 0.5| < policy_margin, or no network is
                             loaded, the threshold rule decides; default 0.05 */
  int32_t filter_degree;  /* neighbour filtering (with IPGC_FORBIDDEN_RESCAN; see `forbidden`):
                             once the worklist is small (filter_start),
                             a node of degree > max(filter_degree, chunk, t1) keeps the list
                             of its still-active neighbours and a bitmap of the colours of
                             its finalised ones, so later rounds read only the active part
                             of its row (same colours; more workspace: about 8 bytes per
                             entry). 0 = default 1024; < 0 = off. Single-graph entry points
                             only; used while every colour is <= 2047. */
  float filter_start;     /* filtering starts at the first round r >= 3 whose worklist has at
                             most filter_start * n nodes of mean degree above the filter
                             degree; 0 = default 1/32 */
  int32_t worklist;       /* IPGC_WORKLIST_KEEP (default): every round pushes the worklist,
                             topology-driven ones too (the paper's hybrid, Sections I and IV);
                             IPGC_WORKLIST_REBUILD: topology-driven rounds only count the
                             active nodes and the first data-driven round after them rebuilds
                             the worklist from the colours (the hybrid of Nasre et al. that the
                             paper compares against, Section I). Same colours either way.
                             REBUILD runs without neighbour filtering and only with the
                             persistent driver (IPGC_ERR_UNSUPPORTED otherwise). */
  int32_t forbidden;      /* how the assignment step of a node of degree > t1 learns the colours
                             of its finalised neighbours (its forbidden colours, Section II-C):
                             IPGC_FORBIDDEN_RESCAN: every round rereads the node's row (the
                             paper's loop; with neighbour filtering);
                             IPGC_FORBIDDEN_PUSH: the node keeps a bitmap of those colours, into
                             which each neighbour ORs its colour once, when it is committed, so
                             a row is read about once in all instead of once per round; a node
                             with several work items also keeps the list of its still-active
                             lower-ID neighbours for its conflict step. Same colours; about 12
                             more bytes of workspace per entry and 12 per node; needs the
                             persistent driver (IPGC_ERR_UNSUPPORTED otherwise); forced, it
                             turns neighbour filtering off;
                             rounds that start with a colour above 2046 committed rescan; a
                             graph without a node of degree > t1 is coloured by rescanning.
                             IPGC_FORBIDDEN_AUTO (0, default): PUSH with the persistent driver
                             when the rows of the nodes of degree > t1 hold at least half of
                             the entries (checked on the device before round 1), else RESCAN
                             (with neighbour filtering as filter_degree says; the workspace
                             holds what both need); RESCAN with the host-loop driver. */
} ipgc_options;

#define IPGC_WORKLIST_KEEP 0
#define IPGC_WORKLIST_REBUILD 1

#define IPGC_FORBIDDEN_AUTO 0
#define IPGC_FORBIDDEN_RESCAN 1
#define IPGC_FORBIDDEN_PUSH 2

/* Fill *opt with the defaults listed above. */
IPGC_API void ipgc_options_default(ipgc_options* opt);

/* Message for a status code (static storage, never NULL). */
IPGC_API const char* ipgc_strerror(int status);

/*
 * Create a context on CUDA device `device`. The context owns the workspace
 * (tentative colours, worklists, control block), grown on demand and reused
 * by later calls. A context must not be used by two host threads at once.
 * Errors: IPGC_ERR_INVALID (bad device), IPGC_ERR_CUDA, IPGC_ERR_OOM.
 */
IPGC_API int ipgc_ctx_create(ipgc_ctx** out, int device);
IPGC_API int ipgc_ctx_destroy(ipgc_ctx* ctx);
/* The last CUDA error code (cudaError_t) seen by the context, 0 if none. */
IPGC_API int ipgc_ctx_cuda_error(const ipgc_ctx* ctx);

/*
 * Bytes of device workspace a colouring of a graph with n nodes and nnz entries
 * needs under options opt (NULL = defaults; the degree thresholds matter)
 * (ipgc_color_ex grows the context's workspace to this size when needed).
 */
IPGC_API size_t ipgc_workspace_size(int32_t n, int64_t nnz, const ipgc_options* opt);

/*
 * Colour one graph (Section II-C's loop with Section IV's hybrid schedule).
 *   rowptr      device pointer, int32[n + 1], rowptr[0] = 0, rowptr[n] = nnz
 *   col         device pointer, int32[nnz], see "Graph input" above
 *   n, nnz      node and entry counts (n >= 0, 0 <= nnz < 2^31)
 *   colors_out  device pointer, int32[n]; receives colours 1..num_colors
 *   stats_out   host pointer or NULL. Non-NULL: the call waits for the stream
 *               and fills the statistics (device-side errors are returned).
 *               NULL: the call only enqueues work and returns IPGC_OK; read
 *               the outcome with ipgc_ctx_last_stats after synchronising.
 *   opt         host pointer or NULL (defaults)
 *   stream      cudaStream_t or NULL
 * ipgc_color is ipgc_color_ex on a per-thread default context for the current
 * device, default options and the legacy default stream.
 * Errors: IPGC_ERR_INVALID (arguments; CSR if opt->validate), IPGC_ERR_OOM,
 * IPGC_ERR_TIMEOUT, IPGC_ERR_NO_CONVERGE, IPGC_ERR_CUDA.
 */
IPGC_API int ipgc_color(const int32_t* rowptr, const int32_t* col, int32_t n, int64_t nnz,
               int32_t* colors_out, ipgc_stats* stats_out);
IPGC_API int ipgc_color_ex(ipgc_ctx* ctx, const int32_t* rowptr, const int32_t* col, int32_t n, int64_t nnz,
                  int32_t* colors_out, ipgc_stats* stats_out, const ipgc_options* opt,
                  void* stream);

/* Statistics of the context's last colouring; waits for its stream. */
IPGC_API int ipgc_ctx_last_stats(ipgc_ctx* ctx, ipgc_stats* stats_out);

/*
 * As ipgc_color_ex, but rowptr, col and colors_out are HOST pointers: the
 * call copies the graph to device buffers held by the context, colours it and
 * copies the colours back, all on `stream`, and returns when they are in
 * colors_out. Pinned host memory makes the copies faster but is not required.
 */
IPGC_API int ipgc_color_host(ipgc_ctx* ctx, const int32_t* rowptr, const int32_t* col, int32_t n,
                    int64_t nnz, int32_t* colors_out, ipgc_stats* stats_out,
                    const ipgc_options* opt, void* stream);

/*
 * Check that a CSR is an input the method is defined on: the undirected graph
 * G = (V, E) of the problem statement (Section II-A), so symmetric (u in row
 * v iff v in row u), with the self-loops and multi-edges removed (Section V),
 * so no entry (v, v) and no duplicate entry; also rowptr[0] == 0, rowptr
 * non-decreasing, rowptr[n] == nnz, every col entry in [0, n) and every row
 * ascending (the layout the colouring kernels read).
 * on_device = 1: rowptr/col are device pointers and kernels check them on
 * the context's stream (ctx may be NULL: current device, default stream;
 * the call waits for the stream); every entry is read once and each
 * undirected pair is looked up once, in the shorter of its two rows.
 * on_device = 0: host pointers, checked on the host. Returns IPGC_OK or
 * IPGC_ERR_INVALID (also for n < 0, nnz outside [0, 2^31) or a NULL
 * pointer), IPGC_ERR_CUDA, IPGC_ERR_OOM.
 */
IPGC_API int ipgc_validate_csr(ipgc_ctx* ctx, const int32_t* rowptr, const int32_t* col, int32_t n,
                      int64_t nnz, int on_device, void* stream);

/*
 * Batched colouring: many independent graphs in one persistent launch. The
 * paper colours one graph per run; this form applies its loop (Section
 * II-C) and hybrid schedule (Section IV) to every graph of a batch, each
 * graph with its own worklists, rounds and mode decisions, so each graph gets
 * exactly the colouring ipgc_color_ex would give it alone. A graph is
 * coloured by a team of k CTAs, k the smallest power of two with
 * k * nnz_per_cta >= its entries, or min(max_team, grid) where that is
 * smaller; teams are gang-scheduled on aligned blocks of CTAs, largest
 * first, and graphs with k = 1 are taken one CTA each from a shared queue. Options in `base` apply
 * to every graph (trace, fin_round, driver, blocks_per_sm and fault_inject
 * are ignored). Unless base.forbidden is IPGC_FORBIDDEN_RESCAN, graphs with a
 * node of degree > t1 are coloured with forbidden-colour bitmaps (a first
 * launch; see ipgc_options.forbidden) and the others by rescanning rows (a
 * second launch, with a schedule of its own).
 */
typedef struct ipgc_batch_options {
  ipgc_options base;     /* defaults as ipgc_options_default, but validate = 0 */
  int32_t max_team;      /* largest team in CTAs, >= 0 (0: the whole grid); default 0 */
  int32_t reserved;
  int64_t nnz_per_cta;   /* entries per CTA of a team, >= 1; default 131072 */
} ipgc_batch_options;

IPGC_API void ipgc_batch_options_default(ipgc_batch_options* opt);

/*
 *   num_graphs   G >= 0
 *   node_off     HOST pointer, int64[G + 1]: graph g has nodes
 *                [node_off[g], node_off[g + 1]) of the concatenation
 *   edge_off     HOST pointer, int64[G + 1]: graph g's entries in col_cat
 *   rowptr_cat   device pointer: graph g's local rowptr (n_g + 1 entries,
 *                values in [0, nnz_g]) starts at rowptr_cat[node_off[g] + g]
 *   col_cat      device pointer: graph g's local neighbour IDs at edge_off[g]
 *   colors_cat   device pointer, int32[node_off[G]]: graph g's colours at
 *                node_off[g]
 *   per_graph_stats  host pointer to G records, or NULL (then the call only
 *                enqueues work on `stream`)
 * The context keeps a batched workspace (about 12 bytes per node, 16 bytes
 * per work item and 256 bytes per large node; with bitmaps also 12 bytes per
 * entry and 4 per node), grown on demand.
 * Returns IPGC_OK or the first per-graph error (IPGC_ERR_INVALID for a bad
 * graph when base.validate is set, IPGC_ERR_TIMEOUT, IPGC_ERR_NO_CONVERGE),
 * IPGC_ERR_OOM, IPGC_ERR_CUDA.
 */
IPGC_API int ipgc_color_batched(ipgc_ctx* ctx, int32_t num_graphs, const int64_t* node_off,
                                const int64_t* edge_off, const int32_t* rowptr_cat,
                                const int32_t* col_cat, int32_t* colors_cat,
                                ipgc_stats* per_graph_stats, const ipgc_batch_options* opt,
                                void* stream);

/*
 * The schedule ipgc_color_batched uses on `grid` CTAs, computed on the host
 * (no device needed). Inputs: n[g], nnz[g] per graph (HOST arrays). Outputs
 * (HOST int32[num_graphs], caller-owned): team[g] = CTAs colouring graph g
 * (0: empty graph, 1: the single-CTA queue); first_cta[g] = first CTA of its
 * aligned block of team[g] CTAs (-1 for team[g] <= 1); seq[g] = position in
 * the gang order of the teams (every CTA runs its team jobs in this order)
 * or in the single-CTA queue (-1 for empty graphs). IPGC_OK or
 * IPGC_ERR_INVALID.
 */
IPGC_API int ipgc_batch_plan(int32_t num_graphs, const int32_t* n, const int64_t* nnz,
                             int32_t grid, int32_t max_team, int64_t nnz_per_cta, int32_t* team,
                             int32_t* first_cta, int32_t* seq);

/*
 * Colouring server with continuous batching (not in the paper: a serving
 * form of Section II-C's loop, whose results are those of colouring each
 * request alone with the batched phases above). Requests are host
 * CSR graphs, copied into pinned staging at submission and queued in order.
 * A scheduler thread admits queued requests while the device arena (one
 * allocation of hbm_budget bytes) has room for the graph, its colours and its
 * working set, copies them to the device, and colours every admitted request
 * in one batched launch whenever one of `inflight` batch slots is free; the
 * slots run concurrently on their own streams, so requests arriving while
 * others are on the GPU start without waiting for them to finish. Each
 * request completes as soon as its own graph is coloured (the kernel writes
 * the result into pinned staging and raises a host-visible flag), not when
 * its batch ends, and its device memory then admits the next requests at
 * once. Each result is the colouring the graph gets alone (the batched
 * phases). Unless batch.base.forbidden is IPGC_FORBIDDEN_RESCAN, the
 * launches colour with forbidden-colour bitmaps (see ipgc_options.forbidden;
 * graphs without a node of degree > t1 rescan in the same launch), and each
 * request's device memory holds its bitmaps and lists (about 12 more bytes
 * per entry and 16 per node). With batch.base.mode = IPGC_MODE_LEARNED the
 * network loaded by ipgc_server_policy_load chooses each round's mode (the
 * threshold rule without one, or where it is unsure).
 */
typedef struct ipgc_server ipgc_server;

typedef struct ipgc_server_options {
  size_t hbm_budget;          /* device arena bytes; default 8 GiB */
  size_t host_budget;         /* pinned staging bytes; default 4 GiB */
  int32_t inflight;           /* concurrent batches, 1..8; default 2 */
  int32_t max_batch_graphs;   /* graphs per launch; default 1024 */
  int32_t max_pending;        /* queued, not yet admitted requests; default 65536 */
  int32_t reserved;
  ipgc_batch_options batch;   /* schedule and mode (base.validate: check each CSR on submit) */
} ipgc_server_options;

typedef struct ipgc_server_counters {
  uint64_t submitted, completed, batches, graphs_in_batches;
  int64_t pending;            /* queued, waiting for device memory */
  int64_t ready;              /* admitted, waiting for a batch slot */
  int32_t running_batches;
  int32_t max_batch;          /* largest batch launched so far */
  int64_t hbm_used, hbm_peak; /* device arena bytes in use / at most */
  int64_t host_used;          /* pinned staging bytes in use */
  int32_t status;             /* IPGC_OK or the error that stopped the server */
  int32_t reserved;
} ipgc_server_counters;

IPGC_API void ipgc_server_options_default(ipgc_server_options* opt);
/* Allocates the arenas and starts the scheduler thread on `device`. */
IPGC_API int ipgc_server_create(ipgc_server** out, int device, const ipgc_server_options* opt);
/*
 * Queue one graph (HOST pointers, copied before the call returns).
 * IPGC_ERR_TOO_LARGE: it can never fit the budgets; IPGC_ERR_BUSY: the
 * queue or the staging is full right now (retry later); IPGC_ERR_INVALID.
 */
IPGC_API int ipgc_server_submit(ipgc_server* srv, const int32_t* h_rowptr, const int32_t* h_col,
                                int32_t n, int64_t nnz, uint64_t* ticket);
/*
 * The same without the copy: the server reads the graph from the caller's
 * arrays when it admits the request, so they must stay valid and unchanged
 * until the ticket completes. Page-locked (pinned) arrays let the copy to the
 * device run asynchronously; pageable ones are copied synchronously.
 */
IPGC_API int ipgc_server_submit_ref(ipgc_server* srv, const int32_t* h_rowptr,
                                    const int32_t* h_col, int32_t n, int64_t nnz,
                                    uint64_t* ticket);
/*
 * IPGC_PENDING while the request runs. Otherwise copies its colours to
 * h_colors (host int32[n], may be NULL), its statistics and its latency
 * (submission to completion, ns; may be NULL), releases the ticket and
 * returns its status; IPGC_ERR_NOT_FOUND for an unknown or released ticket.
 */
IPGC_API int ipgc_server_poll(ipgc_server* srv, uint64_t ticket, int32_t* h_colors,
                              ipgc_stats* stats, int64_t* latency_ns);
/* The next completed ticket (each reported once); IPGC_PENDING after timeout_ns. */
IPGC_API int ipgc_server_next_done(ipgc_server* srv, uint64_t* ticket, uint64_t timeout_ns);
IPGC_API int ipgc_server_query(ipgc_server* srv, ipgc_server_counters* counters);
/*
 * The learned mode switch of the server's launches (see ipgc_policy_load):
 * len = IPGC_MLP_PARAMS host floats, copied into device memory of the
 * server's own; launches that start afterwards use them (those already
 * running keep the network they started with). len = 0 unloads. Used only
 * when the server's batch.base.mode is IPGC_MODE_LEARNED; colours never
 * depend on it. IPGC_ERR_INVALID (wrong length), IPGC_ERR_OOM, IPGC_ERR_CUDA.
 */
IPGC_API int ipgc_server_policy_load(ipgc_server* srv, const float* w, int32_t len);
/* Finishes admitted work, drops queued requests, frees everything. */
IPGC_API int ipgc_server_destroy(ipgc_server* srv);

/*
 * Learned mode switch. A multilayer perceptron 8 -> 16 -> 16 -> 1 (tanh
 * hidden units, logistic output) gives the probability that the round runs
 * faster topology-driven than data-driven (Section IV leaves the choice of H
 * to experiment; Section VII asks for a better rule). Parameters, float32,
 * IPGC_MLP_PARAMS of them: W1[16][8], b1[16], W2[16][16], b2[16], w3[16], b3.
 * The 8 inputs of a round are computed from its trace record by
 * ipgc_policy_features (the colouring kernel computes the same values the
 * same way when it runs with IPGC_MODE_LEARNED).
 */
#define IPGC_MLP_INPUTS 8
#define IPGC_MLP_HIDDEN 16
#define IPGC_MLP_PARAMS 433

/* Features of `rounds` trace records (device pointers; feats: float[rounds][8]). */
IPGC_API int ipgc_policy_features(const ipgc_trace_rec* trace, int32_t rounds, int32_t n,
                                  int64_t nnz, float* feats, void* stream);
/* Forward pass: prob[i] = network output for x[i][0..8) (device pointers). */
IPGC_API int ipgc_mlp_forward(const float* w, const float* x, int32_t n, float* prob, void* stream);
/*
 * Loss and gradient of the weighted logistic loss
 *   L = sum_i wt[i] * (softplus(z_i) - y[i] * z_i) / sum_i wt[i]
 * over n samples (device pointers; y in {0, 1}, wt >= 0). grad: float[433],
 * loss: float[1]; scratch: float[434 * n] per-sample terms, summed in a fixed
 * order (the result does not depend on thread timing).
 */
IPGC_API int ipgc_mlp_grad(const float* w, const float* x, const float* y, const float* wt,
                           int32_t n, float* grad, float* loss, float* scratch, void* stream);
/*
 * Full-batch Adam on the device with the kernels above (beta1 0.9, beta2
 * 0.999, eps 1e-8): `epochs` steps from the weights in w_inout (device
 * float[433]), updated in place. loss_out (host, may be NULL) receives the
 * loss before the last step. Scratch comes from the context's workspace.
 */
IPGC_API int ipgc_mlp_train(ipgc_ctx* ctx, const float* x, const float* y, const float* wt,
                            int32_t n, int32_t epochs, float lr, float* w_inout, float* loss_out,
                            void* stream);
/* Copy 433 host floats into the context; IPGC_MODE_LEARNED then uses them. len = 0 unloads. */
IPGC_API int ipgc_policy_load(ipgc_ctx* ctx, const float* w, int32_t len);

/*
 * Schedule autotuners. The paper maps work to threads with Nested
 * Parallelism and tunes nothing per input (Section V); here the mapping's
 * knobs (t1, chunk, block_size and, for batches, max_team and nnz_per_cta)
 * are chosen by timing. The schedule changes speed only, never a
 * colour. Starting from *opt, each knob in turn is set to every candidate
 * value, the colouring is timed (best of `reps`, CUDA events on `stream`) and
 * the fastest value is kept; *opt receives the result and *best_ms (may be
 * NULL) its time. ipgc_autotune times ipgc_color_ex on the given graph
 * (colors_scratch: device int32[n], overwritten); ipgc_batched_autotune times
 * ipgc_color_batched on the batch's first sample_graphs graphs (0 = all),
 * then (with a sample) its choice and the given options on the whole batch,
 * keeping the faster, writing colours to colors_cat. Errors as the timed
 * calls.
 */
IPGC_API int ipgc_autotune(ipgc_ctx* ctx, const int32_t* rowptr, const int32_t* col, int32_t n,
                           int64_t nnz, int32_t* colors_scratch, int32_t reps, ipgc_options* opt,
                           float* best_ms, void* stream);
IPGC_API int ipgc_batched_autotune(ipgc_ctx* ctx, int32_t num_graphs, const int64_t* node_off,
                                   const int64_t* edge_off, const int32_t* rowptr_cat,
                                   const int32_t* col_cat, int32_t* colors_cat,
                                   int32_t sample_graphs, int32_t reps, ipgc_batch_options* opt,
                                   float* best_ms, void* stream);

/*
 * The micro-benchmark of Section III (Listings "Push Kernels" and "Kernel
 * Calls"): the worklist starts as all n nodes and iteration i deactivates
 * the next `count` IDs (node v stays active iff v >= count * (i + 1), the
 * text's reading of the listing), until the worklist is empty, i.e. for
 * ceil(n / count) iterations. Each iteration keeps a worklist:
 *   IPGC_PUSH_WL      Push_WL: iterate over the worklist (data-driven);
 *   IPGC_PUSH_NOWL    Push_NoWL: iterate over all n nodes (topology-driven);
 *   IPGC_PUSH_HYBRID  Push_NoWL while |WL| > switch_wl, then Push_WL.
 * All iterations run in one cooperative launch (the Pipe). Arguments:
 *   n          0 <= n < 2^31 nodes; count >= 1
 *   rec        device pointer to cap records of 4 int64 each, or NULL (cap 0):
 *              record i = {|WL| after iteration i, sum of the IDs in it, the
 *              kernel used (IPGC_PUSH_WL / IPGC_PUSH_NOWL), the iteration's
 *              time in ns (%globaltimer)}; iterations >= cap are not recorded
 *   iterations host pointer (may be NULL): the number of iterations
 * The worklists (2n int32) live in the context's auxiliary buffer. The call
 * synchronises `stream`. Returns IPGC_OK, IPGC_ERR_INVALID, IPGC_ERR_OOM,
 * IPGC_ERR_CUDA or IPGC_ERR_TIMEOUT (a bounded barrier gave up).
 */
#define IPGC_PUSH_WL 0
#define IPGC_PUSH_NOWL 1
#define IPGC_PUSH_HYBRID 2
IPGC_API int ipgc_push_bench(ipgc_ctx* ctx, int64_t n, int32_t count, int32_t mode,
                             int64_t switch_wl, int64_t* rec, int64_t cap, int64_t* iterations,
                             void* stream);

/*
 * Colour one graph without allocating anything (the paper has no counterpart;
 * this exists for callers that cannot allocate device memory when they need
 * a colouring, e.g. code running inside an allocator or memory-pool callback,
 * which must not re-enter the allocator, or a service that works within a
 * budget reserved up front). The CSR is always validated. The colouring is
 * the rescanning one (every round rereads the active nodes' rows) with the
 * default degree bound t1 = 64 fixed and the default work items and
 * threshold rule; colours, rounds, num_colors, rounds_topo and rounds_data
 * equal those of ipgc_color_ex with default options (edges_processed and ns
 * describe this call's own work).
 *   rowptr, col   device pointers as for ipgc_color_ex
 *   n, nnz        at most IPGC_NOALLOC_MAX_N nodes and IPGC_NOALLOC_MAX_NNZ
 *                 entries; larger graphs return IPGC_ERR_TOO_LARGE before any
 *                 CUDA call
 *   colors_out    device pointer, int32[n]
 *   stats_out     host pointer or NULL
 *   stream        cudaStream_t or NULL
 * The call waits for `stream` (after validation and after the colouring) and
 * returns the error the device reported, with or without stats_out.
 * Working memory is one fixed device array inside the library (15,074,048
 * bytes), shared by all calls: calls that overlap on one GPU race and must be
 * serialised by the caller. No cudaMalloc or cudaFree is made. The first call
 * on a device looks up the array's device address, which also loads the
 * library's device code, and the array with it, onto that device if nothing
 * else did (lazy module loading); so make that first call at set-up (an
 * empty graph, n = 0, will do), before any stream capture and before the
 * point where allocating is no longer possible. The device then holds the
 * array until the process exits.
 * Errors: IPGC_ERR_INVALID, IPGC_ERR_TOO_LARGE, IPGC_ERR_TIMEOUT,
 * IPGC_ERR_NO_CONVERGE, IPGC_ERR_CUDA, IPGC_ERR_UNSUPPORTED.
 */
#define IPGC_NOALLOC_MAX_N 524288
#define IPGC_NOALLOC_MAX_NNZ 8388608
IPGC_API int ipgc_color_noalloc(const int32_t* rowptr, const int32_t* col, int32_t n, int64_t nnz,
                                int32_t* colors_out, ipgc_stats* stats_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* IPGC_H */
