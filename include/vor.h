/*
 * vor.h -- C ABI of the GB300 projector-algorithm library (libvor.so).
 *
 * The library computes, on one GPU, the Voronoi diagram of n distinct integer
 * point sites inside a rectangle X = [0,w] x [0,h] and the Delaunay graph
 * restricted to X.  It follows D. Reem, "The projector algorithm: a simple
 * parallel algorithm for computing Voronoi diagrams and Delaunay graphs":
 *
 *   - Definition 2.1 defines the cell R_k of site p_k;
 *   - Theorem 2.2 / eq. (2.1) define the ray endpoint T(p, theta) that every
 *     ray of the method computes;
 *   - Algorithm 1 (Section 4) is the per-cell projector run by the kernels;
 *   - Section 5 defines what is stored per cell (vertices and the lines they
 *     lie on, labelled by neighbour site), Section 6 the Delaunay graph;
 *   - Theorem 8.1(c,d) states that cells are independent, which is how the
 *     work is spread over the GPU.
 *
 * Conventions (all entry points):
 *   - Sites are int32 pairs with 0 < x < w and 0 < y < h (the paper assumes
 *     sites in the interior of X, Section 2), pairwise distinct, and
 *     2 <= w, h <= 2^20 (the bound keeps every exact predicate within
 *     128-bit integers).
 *   - A line of a cell is labelled by the index j >= 0 of the neighbour site
 *     whose bisector carries the edge, or by a side of X:
 *       VOR_SIDE_BOTTOM (-1), VOR_SIDE_RIGHT (-2), VOR_SIDE_TOP (-3),
 *       VOR_SIDE_LEFT (-4).
 *   - Cell k lists the lines carrying an edge of positive length, ordered
 *     counter-clockwise by the polar angle of the edge's outward normal and
 *     starting at the smallest angle in [0, 2 pi).  Vertex i of cell k is the
 *     point shared by edges i and i+1 (cyclically), in float64.
 *   - Delaunay edges are pairs (k, j) with k < j whose cells share an edge of
 *     positive length, ordered by k, then j.
 *   - Every pointer named d_* is device memory of the current CUDA device;
 *     h_* is host memory.  Buffers stay owned by the caller.  All device
 *     work is ordered on the given stream; nothing is launched on another
 *     stream.
 *   - Functions return VOR_OK (0) or a negative VOR_E_* code.  No exception,
 *     abort or device trap crosses this interface.  After an error the output
 *     buffers hold unspecified values.
 */
#ifndef VOR_H
#define VOR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VOR_OK 0
#define VOR_E_INVALID_ARG (-1)   /* null pointer, n < 1, bad option          */
#define VOR_E_SITE_OUTSIDE (-2)  /* a site on or outside the boundary of X   */
#define VOR_E_DUPLICATE (-3)     /* two equal sites                          */
#define VOR_E_BOX_TOO_LARGE (-4) /* w or h outside [2, 2^20]                 */
#define VOR_E_OOM (-5)           /* workspace or output too small / no memory */
#define VOR_E_CAPACITY (-6)      /* a capacity of the build was exceeded     */
#define VOR_E_CUDA (-7)          /* a CUDA runtime call failed               */
#define VOR_E_INTERNAL (-8)      /* an internal consistency check failed     */
#define VOR_E_SCRATCH_LIMIT (-9) /* vor_build_noalloc: n needs more than its static scratch */
#define VOR_E_SERVER_FULL (-10)  /* request larger than a server budget; or submit timed out */
#define VOR_E_TIMEOUT (-11)      /* vor_server_wait: the request is still pending          */
#define VOR_E_CANCELLED (-12)    /* the request was cancelled                              */
#define VOR_PENDING 1            /* vor_server_poll: not finished yet                      */

#define VOR_SIDE_BOTTOM (-1)
#define VOR_SIDE_RIGHT (-2)
#define VOR_SIDE_TOP (-3)
#define VOR_SIDE_LEFT (-4)

typedef struct vor_site { int32_t x, y; } vor_site;
typedef struct vor_box { int32_t w, h; } vor_box;

/* Tuning knobs; vor_opts_default() fills the automatic values. */
typedef struct vor_opts {
    int32_t bucket_side;      /* bucket side s in units of X (Method A.5); 0: automatic     */
    int32_t lanes_per_cell;   /* lanes cooperating on one cell: 1,2,4,8,16,32; 0: automatic */
    int32_t target;           /* sites wanted in the first candidate disc around a site
                                 (its radius follows the local bucket density); 0: 24      */
    int32_t exact_only;       /* 1: skip the float filter, decide every ray exactly      */
    int32_t check_duplicates; /* 1: reject equal sites (VOR_E_DUPLICATE)                  */
    int32_t collect_stats;    /* 1: fill vor_stats (device atomics, slightly slower)      */
    int32_t bucket_load_pct;  /* automatic bucket side: sites per bucket it aims at around
                                 a typical site, in hundredths (25..1600); 0: 600          */
    int32_t share_vertices;   /* a Voronoi vertex belongs to two or three cells (Section 9
                                 notes it is computed three times).  0: every cell computes
                                 it from its owner's lines (the cell of the smallest site
                                 among them), so all copies are bit-identical; 1: only the
                                 owner computes it and the other cells copy it (one extra
                                 kernel; slower on this GPU than computing it again)     */
    int32_t fine_split;       /* adaptive buckets (Section 9 suggests a bucketing structure
                                 fitted to the distribution of the sites): a bucket holding
                                 at least this many sites (4..65536) is divided into F x F
                                 sub-buckets (F = 2..16, about three sites each), which the
                                 thread-per-cell gathers and their first disc's density
                                 estimate use.  0: no sub-buckets (the default; slower on
                                 this GPU for the measured workloads)                     */
    int32_t block_threads;    /* block shape of the thread-per-cell first pass: 32, 64 or
                                 128 threads per block; 0: 64                             */
} vor_opts;

/* Counters of one build (filled when collect_stats = 1). */
typedef struct vor_stats {
    uint64_t rays;             /* endpoint computations (rays shot, Algorithm 1)          */
    uint64_t vertex_tests;     /* "u inside the cell" tests (Algorithm 1)                 */
    uint64_t evals;            /* candidate evaluations of the float filter                */
    uint64_t exact_rays;       /* rays or tests the float filter could not decide         */
    uint64_t annulus_sites;    /* sites checked by the security-radius certificate        */
    uint64_t reruns;           /* cells recomputed after the certificate added sites      */
    uint64_t deferred;         /* cells handed to the large-cell kernel                   */
    uint64_t candidates;       /* candidate sites staged, summed over cells                */
    uint64_t max_edges;        /* largest e_k                                              */
    uint64_t widenings;        /* certificate steps that grew the tested region            */
    uint64_t evals_first_pass; /* the part of evals done by the first thread-per-cell pass */
    uint64_t rays_first_pass;  /* the part of rays shot by the first thread-per-cell pass  */
    uint64_t evals_second_pass;/* the part of evals done by the second thread-per-cell pass*/
    uint64_t third_pass_cells; /* cells handed to the thread-per-cell flower passes        */
    uint64_t medium_cells;     /* cells handed to the warp-per-cell medium tier            */
    uint64_t large_cells;      /* cells handed on to the block-per-cell tier               */
    uint64_t global_cells;     /* of those, cells too large for its shared-memory mode     */
    uint64_t divided_buckets;  /* buckets divided into sub-buckets (adaptive buckets)      */
} vor_stats;

/* Device output buffers, allocated by the caller with the capacities below:
 *   cell_ptr  int64[n + 1]             CSR offsets of cells into the edge arrays
 *   edge_label int32[edge_cap]         line labels, canonical order per cell
 *   vx, vy    double[edge_cap]         vertex coordinates
 *   del_edge  int32[2 * del_cap]       Delaunay pairs (k, j)
 *   totals    int64[2]                 written: total edges, total Delaunay edges
 * edge_cap >= vor_edge_capacity(n) and del_cap >= vor_delaunay_capacity(n)
 * always suffice (the paper bounds sum_k e_k by (|X_e| + 6) n = 10 n for a
 * rectangle, Lemma NodesO(n), and the Delaunay graph by 3n - 6 edges). */
typedef struct vor_out {
    int64_t *cell_ptr;
    int32_t *edge_label;
    double *vx, *vy;
    int32_t *del_edge;
    int64_t *totals;
    int64_t edge_cap, del_cap;
} vor_out;

/* Fill opts with the defaults (automatic bucket size, lanes and disc size,
 * filter on, duplicate check on, statistics off). */
void vor_opts_default(vor_opts *opts);

/* Capacities that always suffice for n sites (see vor_out). */
int64_t vor_edge_capacity(int64_t n);
int64_t vor_delaunay_capacity(int64_t n);

/* Bytes of device workspace vor_build_async needs for n sites in box with
 * these options (opts may be NULL for the defaults).  Returns -1 on invalid
 * arguments. */
int64_t vor_workspace_bytes(int64_t n, vor_box box, const vor_opts *opts);

/* Build the diagram of n sites d_sites[0..n) (device, int32 pairs) in X.
 *
 * d_workspace: ws_bytes >= vor_workspace_bytes(n, box, opts) bytes of device
 * memory, 256-byte aligned, owned by the caller and not used by anything else
 * until the stream reaches the end of this call's work.
 * out: caller-allocated device buffers (see vor_out).
 * stream: a cudaStream_t (NULL for the legacy default stream).
 *
 * Asynchronous: launches the kernels on the stream and returns without
 * waiting, so validation errors found on the device (VOR_E_SITE_OUTSIDE,
 * VOR_E_DUPLICATE, VOR_E_CAPACITY) are reported by vor_status() after the
 * stream has been synchronised.  Argument errors are returned at once.
 * No memory is allocated; nothing waits on the host. */
int vor_build_async(const vor_site *d_sites, int64_t n, vor_box box, const vor_opts *opts,
                    void *d_workspace, int64_t ws_bytes, const vor_out *out, void *stream);

/* Status of the last vor_build_async that used this workspace: VOR_OK or a
 * device-detected error.  Copies the workspace's 256-byte header to the host
 * on the stream and waits for that stream only (no device-wide
 * synchronisation).  stats (may be NULL) receives the counters. */
int vor_status(const void *d_workspace, void *stream, vor_stats *stats);

/* Synchronous convenience form: allocates workspace and worst-case output
 * with cudaMalloc, builds, waits, and returns the outputs
 * (owned by the caller, free with vor_free_result).  *n_edges and *n_del
 * receive the totals.  The pointers in *out are device pointers. */
int vor_build(const vor_site *d_sites, int64_t n, vor_box box, const vor_opts *opts,
              void *stream, vor_out *out, int64_t *n_edges, int64_t *n_del, vor_stats *stats);
int vor_free_result(vor_out *out, void *stream);

/* End-to-end form with host buffers: copies h_sites to the device, builds,
 * and copies the results back into caller-allocated host arrays
 * (h_cell_ptr[n+1], h_edge_label/h_vx/h_vy[edge_cap], h_del_edge[2*del_cap]).
 * d_workspace/ws_bytes as for vor_build_async; d_scratch must hold
 * vor_host_scratch_bytes(n) bytes of device memory for the staged copies.
 * Returns after the results are on the host. */
int64_t vor_host_scratch_bytes(int64_t n);
int vor_build_host(const vor_site *h_sites, int64_t n, vor_box box, const vor_opts *opts,
                   void *d_workspace, int64_t ws_bytes, void *d_scratch, int64_t scratch_bytes,
                   int64_t *h_cell_ptr, int32_t *h_edge_label, double *h_vx, double *h_vy,
                   int32_t *h_del_edge, int64_t edge_cap, int64_t del_cap,
                   int64_t *n_edges, int64_t *n_del, void *stream);

/* Stage timing, off by default.  When enabled, vor_build_async records a
 * CUDA event on its stream before and after each stage; vor_stage_ms then
 * waits for the last event and writes the device milliseconds of the last
 * timed build: ms[0] planning and bucketing (density probe, validation,
 * count, scan, scatter, duplicate check), ms[1] the candidate gather of the
 * first thread-per-cell pass, ms[2] that pass's projector kernel, ms[3] the
 * second pass (gather and projector), ms[4] the large-cell pass, ms[5]
 * compaction (two scans and the CSR/Delaunay kernel).  With lanes_per_cell
 * > 1, ms[2] is the multi-lane pass and ms[1], ms[3] are zero.  Returns the
 * number of values written (<= max_stages) or a negative VOR_E_* code.  One
 * process-wide set of events on the current device: meant for benchmarking
 * one build at a time.  A build captured into a CUDA graph while timing is
 * enabled records the events at every replay (external event records). */
int vor_stage_timing(int enable);
int vor_stage_ms(float *ms, int max_stages);

/* Build without allocating any device memory.
 *
 * The paper has no counterpart of this entry point; it serves callers that
 * cannot allocate device memory when they need a diagram, such as a plug-in
 * inside a host application whose framework owns the whole device memory
 * pool, or a real-time deployment that forbids device allocation after
 * start-up.
 *
 * The caller provides the sites (d_sites, as for vor_build_async) and the
 * output buffers (out, as for vor_build_async).  The workspace is a static
 * device array of VOR_NOALLOC_SCRATCH_BYTES (64 MiB) inside the library; it
 * occupies that memory on every GPU where it has been loaded until the
 * process exits.  n must satisfy vor_workspace_bytes(n, box, opts) <=
 * VOR_NOALLOC_SCRATCH_BYTES (up to 85,228 sites in a 2^20 x 2^20 box with the
 * default options); larger n is rejected with VOR_E_SCRATCH_LIMIT before any
 * work is launched.  No cudaMalloc, cudaFree or other allocating routine is called.
 *
 * Every call looks up the array's device address with cudaGetSymbolAddress
 * in the context current on the calling thread (an address is valid only in
 * its context; after cudaDeviceReset the array is loaded again elsewhere).
 * The first call in a context may load the library's module that holds the
 * array, which reserves its memory: make that first call before any stream
 * capture.  Every call shares the one array,
 * and the build clears on the stream what must start at zero, so calls that
 * overlap on the GPU (on different streams or from different threads) race
 * and corrupt each other: serialise them.
 *
 * Synchronous: launches the build on the stream, waits for the stream and
 * returns VOR_OK or the first error, including the errors vor_build_async
 * leaves to vor_status (VOR_E_SITE_OUTSIDE, VOR_E_DUPLICATE,
 * VOR_E_CAPACITY).  out->totals receives the totals. */
#define VOR_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)
int vor_build_noalloc(const vor_site *d_sites, int64_t n, vor_box box, const vor_opts *opts,
                      const vor_out *out, void *stream);

/* ---- Batches: many independent point sets in one build -------------------
 *
 * The paper computes one diagram at a time; the cells of a diagram are
 * independent (Theorem 8.1(c,d)), and so are the cells of different
 * diagrams.  A batch runs S independent sets through one pass of the
 * pipeline (one launch per stage for the whole batch), which is what makes
 * thousands of small sets cheap: a set of a few hundred sites cannot fill
 * the GPU on its own.
 *
 * Set j (0 <= j < S) is the sites d_sites[set_ptr[j] .. set_ptr[j+1]) in the
 * box boxes[j]; set_ptr[0] = 0, set_ptr is non-decreasing (empty sets are
 * allowed) and N = set_ptr[S] <= 2^27.  Each set follows the conventions of
 * a single build in its own box, with labels LOCAL to the set: a cell of set
 * j lists neighbour indices in [0, n_j) or sides, and its Delaunay pairs
 * (k, l), k < l, are local indices too.
 *
 * Outputs are concatenated over the sets (same vor_out buffers):
 *   cell_ptr int64[N + 1]: the cells of set j are cell_ptr[set_ptr[j] ..
 *     set_ptr[j+1]] (offsets into the shared edge arrays);
 *   edge_label, vx, vy: capacity >= vor_batch_edge_capacity(N, S);
 *   del_edge: capacity >= vor_batch_delaunay_capacity(N, S) pairs, the pairs
 *     of set j at del_edge[2 * d_del_set_ptr[j] .. 2 * d_del_set_ptr[j+1]);
 *   d_del_set_ptr int64[S + 1] (device, caller-allocated): written.
 *   totals: total edges and total Delaunay pairs of the batch.
 *
 * Both the host and the device copies of set_ptr and boxes are required:
 * the host copies size the workspace and the launches, the device copies
 * feed the kernels without a host-to-device copy (so the build can be
 * captured into a CUDA graph).  They must hold the same values; a
 * difference that the device detects is reported as VOR_E_INVALID_ARG by
 * vor_status.  An error (a site outside its box, a duplicate inside a set,
 * a capacity limit) fails the whole batch.  A single build is the batch of
 * one set. */
int64_t vor_batch_edge_capacity(int64_t n_total, int32_t n_sets);
int64_t vor_batch_delaunay_capacity(int64_t n_total, int32_t n_sets);
int64_t vor_batch_workspace_bytes(const int64_t *h_set_ptr, int32_t n_sets, const vor_box *h_boxes,
                                  const vor_opts *opts);
int vor_build_batch_async(const vor_site *d_sites, const int64_t *d_set_ptr,
                          const int64_t *h_set_ptr, int32_t n_sets, const vor_box *d_boxes,
                          const vor_box *h_boxes, const vor_opts *opts, void *d_workspace,
                          int64_t ws_bytes, const vor_out *out, int64_t *d_del_set_ptr,
                          void *stream);

/* Autotuner.  Builds the batch once with each of the n_candidates option
 * sets (one untimed build, then reps timed builds, CUDA events on the
 * stream) and writes the mean device milliseconds of each to ms[] (a
 * candidate whose build fails gets +infinity) and the index of the fastest
 * to *best.  The arguments are those of vor_build_batch_async;
 * ws_bytes must cover vor_batch_workspace_bytes for every candidate.
 * vor_autotune_grid writes the default candidates (lanes per cell and block
 * shape: one thread per cell in blocks of 32, 64 or 128 threads, or 8 lanes
 * per cell; x disc size x bucket load: 36 in all) into cand[0..max) and
 * returns how many it wrote.
 * Synchronous; returns VOR_OK or an argument error. */
int32_t vor_autotune_grid(vor_opts *cand, int32_t max);
int vor_autotune_batch(const vor_site *d_sites, const int64_t *d_set_ptr, const int64_t *h_set_ptr,
                       int32_t n_sets, const vor_box *d_boxes, const vor_box *h_boxes,
                       const vor_opts *candidates, int32_t n_candidates, int32_t reps,
                       void *d_workspace, int64_t ws_bytes, const vor_out *out,
                       int64_t *d_del_set_ptr, void *stream, int32_t *best, float *ms);

/* ---- Serving: a request server with continuous batching ------------------
 *
 * The paper has no counterpart; this is the serving driver around the batch
 * build.  A server owns one device block (its HBM budget), one pinned host
 * block, a few CUDA streams and one dispatcher thread.  Clients submit point
 * sets from host memory at any time and collect their diagrams later:
 *
 *   - Admission.  A submitted request (its sites copied into the pinned
 *     block) waits in arrival order.  Whenever a stream is free, the
 *     dispatcher forms a wave from the longest prefix of waiting requests
 *     that fits the wave limits and the largest free part of the device
 *     block (workspace, sites and worst-case outputs of the batch build),
 *     and launches it: copies in, vor_build_batch_async, status out.
 *     Requests that arrive while waves run join the next wave (continuous
 *     batching); waves on different streams overlap on the GPU.
 *   - Completion.  When a wave's build has finished, its exact result sizes
 *     are read, a host result block of that size is taken from the pinned
 *     block, the results are copied into it and the device memory is freed.
 *   - Errors.  A wave that fails (for instance a site outside its box) is
 *     split: its requests run again one per wave, so only the faulty request
 *     reports the error.  A request larger than either budget is refused at
 *     submission (VOR_E_SERVER_FULL).
 *
 * Results stay valid (host pointers into the pinned block) until
 * vor_server_release.  All functions are thread-safe; CUDA work runs on the
 * dispatcher thread only, on the device current at vor_server_create. */
typedef struct vor_server vor_server;

typedef struct vor_server_config {
    int64_t device_bytes;       /* HBM budget, allocated once at creation          */
    int64_t host_bytes;         /* pinned host memory for staged sites and results  */
    int32_t max_inflight;       /* waves on the GPU at once (one stream each), >= 1 */
    int32_t max_wave_requests;  /* requests per wave, >= 1 (1: no batching)         */
    int64_t max_wave_sites;     /* sites per wave (a larger single request runs alone) */
    vor_opts opts;              /* build options of every wave                      */
    int32_t fail_host_alloc_at; /* fault injection for tests: the k-th result-block
                                   allocation fails (0: never)                      */
} vor_server_config;

typedef struct vor_request_result {
    int32_t status;             /* VOR_OK, VOR_PENDING or a VOR_E_* code             */
    int32_t wave_requests;      /* requests in the wave that built it                */
    int64_t n, n_edges, n_del;
    const int64_t *cell_ptr;    /* host: n + 1 offsets into the edge arrays          */
    const int32_t *edge_label;  /* host: n_edges labels (indices local to the request) */
    const double *vx, *vy;      /* host: n_edges vertices                            */
    const int32_t *del_edge;    /* host: 2 * n_del                                   */
    double t_submit, t_start, t_done;   /* seconds on the server clock (vor_server_now) */
} vor_request_result;

typedef struct vor_server_stats {
    int64_t submitted, completed, failed, cancelled, waves, split_waves, pending, inflight;
    int64_t max_wave_requests_seen, device_free, device_largest_free, host_free;
    int64_t reserved[4];
} vor_server_stats;

void vor_server_config_default(vor_server_config *cfg);
int vor_server_create(const vor_server_config *cfg, vor_server **out);
/* Copies the n sites into the server (waits up to timeout_s seconds for room
 * in the pinned block, else VOR_E_SERVER_FULL) and returns a ticket. */
int vor_server_submit(vor_server *s, const vor_site *h_sites, int64_t n, vor_box box,
                      double timeout_s, uint64_t *ticket);
/* VOR_PENDING while the request runs; else its final status, with res filled. */
int vor_server_poll(vor_server *s, uint64_t ticket, vor_request_result *res);
/* Waits up to timeout_s seconds; VOR_E_TIMEOUT if the request is still pending. */
int vor_server_wait(vor_server *s, uint64_t ticket, double timeout_s, vor_request_result *res);
/* A waiting request is dropped at once; a running one finishes on the GPU
 * and its result is discarded.  The ticket's status becomes VOR_E_CANCELLED. */
int vor_server_cancel(vor_server *s, uint64_t ticket);
/* Frees the ticket and its result (after a final status). */
int vor_server_release(vor_server *s, uint64_t ticket);
int vor_server_statistics(vor_server *s, vor_server_stats *st);
double vor_server_now(const vor_server *s);
/* Stops the dispatcher after the running waves, frees everything. */
int vor_server_destroy(vor_server *s);

/* The vertex-coordinate conversion of the compaction kernel on its own:
 * d_out[i] = d_num[i] / d_den[i] in float64 for n pairs (device arrays).
 * A vertex of a cell is stored as p + N / D with exact integers (Section 5
 * stores vertices; the meeting point of two lines of Section 3); the
 * library writes its float64 coordinate as this quotient of two integers.
 * Domain: 0 <= num < 2^63, 0 < den < 2^44, num / den < 2^21; outside it
 * the result is NaN.  Error at most 2^-42 q + 2^-39 for the exact quotient
 * q, and integer quotients are exact.  Asynchronous on the stream. */
int vor_vertex_quotients(const int64_t *d_num, const uint64_t *d_den, int64_t n, double *d_out,
                         void *stream);

/* Number of kernels this library has launched in this process (all builds,
 * all devices; a captured CUDA graph's replays are not counted). */
int64_t vor_kernel_launches(void);

/* Human-readable text of a VOR_* code. */
const char *vor_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* VOR_H */
