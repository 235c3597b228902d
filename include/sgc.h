/*
 * sgc.h -- cluster-wise Gustavson SpGEMM over CSR_Cluster, GB300 (sm_103a).
 *
 * C ABI of libsgc.so.  Every function returns an int status (SGC_OK on
 * success); sgc_last_error() gives a message for the calling thread's last
 * failure.
 *
 * Conventions that hold for every entry point below:
 *  - Matrix arrays, workspaces and output arrays are DEVICE pointers on the
 *    current CUDA device, allocated and owned by the caller; the library never
 *    frees or keeps them after the call returns (CSR_Cluster keeps the
 *    caller's perm / cluster_ptr pointers by reference for the matrix's life).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls enqueue their kernels on it and return without waiting,
 *    except calls documented as "synchronises", which wait for the stream
 *    because they return a count to the host.
 *  - Sizes come from count-then-fill: a *_workspace_size or *_count call says
 *    how much to allocate, the caller allocates, the fill call writes.
 *  - CSR inputs: int64 row pointer (nrows+1, row_ptr[0] = 0), int32 column
 *    ids sorted ascending and unique within each row, 0 <= col < ncols,
 *    values of the matrix's dtype.  A and B of one product share a dtype.
 *    With sgc_options.validate = 1 these are checked on the device and a
 *    violation returns SGC_DEVICE_CHECK_FAILED; otherwise they are trusted.
 *  - Output C is CSR in A's ORIGINAL row order, columns sorted within each
 *    row, structural entries whose value cancels to zero kept (the symbolic
 *    structure of Sec. 2.2).  FP32 products are accumulated in FP64 and
 *    rounded once; FP64 accumulates in ascending k per (i, j), without FMA
 *    unless sgc_options.fused_fma = 1, except rows computed row by row with
 *    more than SGC_WARP_ROW_OUTPUTS outputs; int64 wraps modulo 2^64.
 *  - Errors: SGC_INVALID_ARG (null pointer, negative or inconsistent size),
 *    SGC_UNSUPPORTED (dtype mismatch, cluster larger than 32 rows),
 *    SGC_WORKSPACE_TOO_SMALL, SGC_CUDA_ERROR (a CUDA call failed; the CUDA
 *    error string is in sgc_last_error), SGC_DEVICE_CHECK_FAILED (a device
 *    check failed: bad input or an internal invariant), SGC_DEVICE_TIMEOUT (a
 *    bounded device-side wait gave up).  On any error, outputs are undefined.
 */
#ifndef SGC_H_
#define SGC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SGC_ABI_VERSION 2

enum {
  SGC_OK = 0,
  SGC_INVALID_ARG = 1,
  SGC_UNSUPPORTED = 2,
  SGC_WORKSPACE_TOO_SMALL = 3,
  SGC_CUDA_ERROR = 4,
  SGC_DEVICE_CHECK_FAILED = 5,
  SGC_DEVICE_TIMEOUT = 6
};

/* value types */
enum { SGC_F32 = 0, SGC_F64 = 1, SGC_I64 = 2 };

/* CSR_Cluster value layouts (Sec. 3.1, "Clustered matrix format") */
enum {
  SGC_LAYOUT_PADDED = 0, /* placeholders kept: value of row l, union column t at val_ptr[c] + t*K_c + l */
  SGC_LAYOUT_MASKED = 1  /* placeholders dropped: values in (t, l ascending over set mask bits) order */
};

/* How kernels fetch B rows.  BULK: the cluster kernels copy them into shared
 * memory with 1D bulk async copies (cp.async.bulk) completing on an mbarrier,
 * and the warp-per-cluster and row kernels prefetch them into L2 with 1D bulk
 * prefetches; LDG: plain loads only. */
enum {
  SGC_STAGING_AUTO = 0, /* BULK when B's col/val base pointers are 16-byte aligned, else LDG */
  SGC_STAGING_BULK = 1,
  SGC_STAGING_LDG = 2
};

/* Rows computed row by row (the row-wise method, and rows of clusters too
 * large for the cluster kernel) use one warp and a per-warp hash table of at
 * most 1024 slots filled to at most min(load_pct, 66)% (numeric), that is up
 * to SGC_WARP_ROW_OUTPUTS outputs at the default load_pct; above that one CTA
 * and a CTA-wide hash table updated with shared-memory atomics; above
 * SGC_HEAVY_ROW_OUTPUTS outputs (4x that many possible outputs in the
 * symbolic phase) a heavy-row CTA with a dense accumulator over column
 * windows, also with atomics.  FP64 values of rows with more outputs than
 * the warp tables take therefore depend on the order of atomic adds, within
 * the FP64 bound; int64 stays exact. */
#define SGC_WARP_ROW_OUTPUTS 675
#define SGC_HEAVY_ROW_OUTPUTS 6144

/* CSR matrix (Sec. 2.1: row-id / col-id / value arrays). */
typedef struct sgc_csr {
  int64_t nrows, ncols, nnz;
  int64_t* row_ptr; /* device, nrows+1 */
  int32_t* col;     /* device, nnz */
  void* val;        /* device, nnz values of dtype */
  int32_t dtype;    /* SGC_F32 / SGC_F64 / SGC_I64 */
  int32_t reserved;
} sgc_csr;

/* CSR_Cluster matrix (Sec. 3.1): rows merged into clusters of K_c <= 32 rows;
 * per cluster the sorted union of the rows' column ids, a presence mask per
 * union column (bit l: row l of the cluster has an entry there), and the
 * values grouped by column with placeholders (PADDED) or without (MASKED).
 * Original row ids are implicit: position p = cluster_ptr[c] + l holds
 * original row perm[p]. */
typedef struct sgc_csr_cluster {
  int64_t nrows, ncols;        /* shape of A */
  int64_t nclusters;
  int64_t nucols;              /* total union columns = ucol_ptr[nclusters] */
  int64_t nvals;               /* value slots = val_ptr[nclusters] */
  int32_t layout;              /* SGC_LAYOUT_* */
  int32_t dtype;
  const int32_t* perm;         /* device, nrows: position -> original row (a permutation) */
  const int64_t* cluster_ptr;  /* device, nclusters+1: cluster c = positions [cluster_ptr[c], cluster_ptr[c+1]) */
  int64_t* ucol_ptr;           /* device, nclusters+1 */
  int32_t* ucol;               /* device, nucols: sorted union column ids per cluster */
  uint32_t* mask;              /* device, nucols */
  int64_t* val_ptr;            /* device, nclusters+1 */
  void* val;                   /* device, nvals */
} sgc_csr_cluster;

typedef struct sgc_options {
  int32_t staging;          /* SGC_STAGING_*; default AUTO */
  int32_t validate;         /* 1: check CSR / CSR_Cluster invariants on the device; default 0 */
  int32_t stage_elems;      /* B elements per staging buffer, 0 = default (2048 numeric, 4096 symbolic) */
  int32_t max_warps;        /* warps (cluster rows in flight) per CTA, 0 = default 8; 1..8 */
  int32_t load_pct;         /* hash table fill limit in percent, 0 = default 75; 25..90 */
  int32_t fused_fma;        /* FP64 values: 1 = accumulate with fused multiply-add (one rounding per
                               term; within the FP64 bound, not bit-identical to separate rounding);
                               0 (default) = product and sum rounded separately.  FP32 inputs always
                               use the fused form: their FP64 products are exact, so it changes nothing. */
  int32_t cluster_load_pct; /* fill limit of the numeric cluster kernel's column table, in percent of its
                               slots; 0 = default 50; 20..75.  Lower: fewer probes, more shared memory. */
  int32_t cluster_kernel;   /* numeric phase: 0 (default) = warp groups for every cluster; 1 = one warp
                               per cluster (B rows prefetched into L2 and streamed through a small
                               shared-memory ring) where the cluster's working set fits in 16 KB,
                               warp groups otherwise */
  int32_t wait_polls;       /* polls of a bounded device-side wait on an mbarrier (the cluster kernels'
                               bulk copies) before it gives up and the call reports SGC_DEVICE_TIMEOUT;
                               0 = default (2^22 polls, about 0.3 s); < 0 = give up without polling, which
                               exercises the timeout path.  After giving up, a kernel waits (with the
                               default limit) for the copies it has in flight before it returns. */
  int32_t accumulator;      /* cluster kernels' accumulator: 0 (default) = a shared-memory hash table of the
                               cluster's output columns, ranked in column order; 1 = dense where it fits: a
                               cluster whose output columns span at most SGC_DENSE_SPAN_MAX columns
                               (smallest to largest column of the B rows it touches) and whose dense
                               working set fits shared memory accumulates into per-row arrays over that
                               span with presence bits (no hashing, no ranking); other clusters use the
                               hash table */
  int32_t spread_max;       /* numeric phase: a cluster whose output-column union times its row count is
                               more than spread_max times its rows' total output count (its per-row
                               accumulators would stay mostly empty) has its rows computed by the row
                               kernels; 0 = default 3; < 0 = never (every cluster that fits shared memory
                               runs in the cluster kernels) */
  int32_t count_staged;     /* 1: the warp-group cluster kernels add the bytes they stage to two counters
                               kept in the workspace (sgc_workspace_counters): B column ids copied into
                               shared memory (whole 16-byte copy windows) and B values read through L2.
                               Costs an atomic per cluster; 0 (default) = off */
  int32_t reserved[4];
} sgc_options;

#define SGC_DENSE_SPAN_MAX 4096

/* Version of this ABI (SGC_ABI_VERSION). */
int sgc_abi_version(void);

/* Number of CUDA kernels the library has launched in this process so far
 * (all threads; a monotone counter for reporting launch counts). */
long long sgc_kernel_launches(void);

/* Message for the calling thread's last failed call ("" if none).  The
 * pointer stays valid until the thread's next call into the library. */
const char* sgc_last_error(void);

/* Fills *opt with the defaults. */
int sgc_default_options(sgc_options* opt);

/* Measured throughput of the FP64 pipe, the arithmetic floor of the numeric
 * phase (one multiply and one add per multiply-add of C = A*B, or one fused
 * multiply-add with sgc_options.fused_fma = 1).  op 0: multiply, 1: add,
 * 2: fused multiply-add.  Runs independent dependency chains on every SM of
 * the current device, `iters` rounds of 16 operations per thread, after one
 * untimed run; *gops_host receives operations (one per lane per
 * instruction) per second / 1e9, timed with CUDA events on `stream`.  sink: a
 * device double the kernel may write.  Synchronises. */
int sgc_fp64_rate(int32_t op, int32_t iters, double* sink, double* gops_host, void* stream);

/* Reads the staging counters kept in a spgemm or learned workspace (see
 * sgc_options.count_staged) into counters_host[0] (bytes of B column ids
 * copied into shared memory) and counters_host[1] (bytes of B values read
 * through L2), summed over every call since they were last cleared; clear = 1
 * zeroes them afterwards.  A new workspace's counters are undefined until
 * cleared.  Synchronises.  SGC_INVALID_ARG on a NULL pointer. */
int sgc_workspace_counters(void* ws, size_t ws_bytes, uint64_t* counters_host, int32_t clear, void* stream);

/* Reads and clears the device status word kept in a spgemm workspace
 * (a failed device check or timeout in an asynchronous call such as
 * spgemm_numeric).  Synchronises.  Returns SGC_OK or the recorded error. */
int sgc_workspace_status(void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * CSR_Cluster construction (Sec. 3.1; A_CSR_CLUSTER(A_CSR, clusters) at the
 * end of Algorithms 2 and 3).
 *
 * csr_cluster_build_count: for clusters given by perm / cluster_ptr over the
 * rows of A (CSR), writes ucol_ptr[0..nclusters] (prefix of union sizes) and
 * val_ptr[0..nclusters] (prefix of value slots for `layout`), both device
 * int64 arrays of nclusters+1 owned by the caller, and returns the totals in
 * *nucols_host and *nvals_host.  ws: device workspace of at least
 * csr_cluster_build_workspace_size(nclusters) bytes.  Checks on the device
 * that perm is a permutation and every cluster has 1..32 rows
 * (SGC_DEVICE_CHECK_FAILED otherwise).  Synchronises.
 * ------------------------------------------------------------------------- */
int csr_cluster_build_workspace_size(int64_t nrows, int64_t nclusters, size_t* bytes);
int csr_cluster_build_count(const sgc_csr* A, const int32_t* perm, const int64_t* cluster_ptr,
                            int64_t nclusters, int32_t layout, int64_t* ucol_ptr, int64_t* val_ptr,
                            int64_t* nucols_host, int64_t* nvals_host, void* ws, size_t ws_bytes,
                            void* stream);

/* csr_cluster_build_count_noalloc: the same counting step as
 * csr_cluster_build_count, for callers that cannot allocate device memory (an
 * application whose allocator owns all device memory, a loop that must not
 * risk an allocation's implicit synchronisation, a tool that accounts for
 * every byte).  The paper has no counterpart; it is a convenience of this
 * library.  It takes no workspace: its scratch (about 16 MiB) is one static
 * device array inside the library, present on every GPU that loads the
 * library until the process exits.  Inputs above SGC_NOALLOC_MAX_ROWS rows or
 * clusters are rejected with SGC_INVALID_ARG.  The first call on a device
 * looks up the array's address (cudaGetSymbolAddress) with that device
 * current; make it before any stream capture.  All calls share the array
 * (cleared at the start of each call): calls that overlap on the GPU race and
 * must be serialised by the caller.  Synchronises; calls no allocator. */
#define SGC_NOALLOC_MAX_ROWS 4194304
int csr_cluster_build_count_noalloc(const sgc_csr* A, const int32_t* perm, const int64_t* cluster_ptr,
                                    int64_t nclusters, int32_t layout, int64_t* ucol_ptr, int64_t* val_ptr,
                                    int64_t* nucols_host, int64_t* nvals_host, void* stream);

/* csr_cluster_build: fills out->ucol, out->mask and out->val (arrays of
 * out->nucols / out->nucols / out->nvals elements allocated by the caller)
 * from A.  out must carry nrows, ncols, nclusters, nucols, nvals, layout,
 * dtype, perm, cluster_ptr, ucol_ptr and val_ptr as returned by
 * csr_cluster_build_count for the same inputs.  Asynchronous. */
int csr_cluster_build(const sgc_csr* A, sgc_csr_cluster* out, void* stream);

/* ---------------------------------------------------------------------------
 * Cluster-wise SpGEMM C = A * B, A in CSR_Cluster (Algorithm 1,
 * ClusterWise_SpGEMM; Sec. 3.1 "Access pattern"): each cluster is one unit of
 * work; every B row k in the cluster's column union is staged in shared
 * memory once and applied to every row of the cluster that has a_lk.
 * Split into the symbolic and numeric phases of Sec. 2.2.
 *
 * spgemm_workspace_size: bytes of device workspace the two calls need for
 * these shapes (independent of values; the same workspace may serve both).
 *
 * spgemm_symbolic: writes C's row pointer c_row_ptr[0..A.nrows] (device,
 * int64, caller-owned, in original row order) and, when c_nnz_host is not
 * NULL, stores nnz(C) there and synchronises; with c_nnz_host NULL it is
 * asynchronous and nnz(C) is c_row_ptr[nrows] on the device.
 *
 * spgemm_numeric: C->row_ptr must hold the symbolic result; writes C->col and
 * C->val (nnz(C) elements each, caller-allocated, dtype = A's).  Asynchronous;
 * device-side failures are reported by sgc_workspace_status.
 * opt may be NULL (defaults).
 * ------------------------------------------------------------------------- */
int spgemm_workspace_size(const sgc_csr_cluster* A, const sgc_csr* B, const sgc_options* opt,
                          size_t* bytes);
int spgemm_symbolic(const sgc_csr_cluster* A, const sgc_csr* B, int64_t* c_row_ptr,
                    int64_t* c_nnz_host, void* ws, size_t ws_bytes, const sgc_options* opt,
                    void* stream);
int spgemm_numeric(const sgc_csr_cluster* A, const sgc_csr* B, sgc_csr* C, void* ws,
                   size_t ws_bytes, const sgc_options* opt, void* stream);

/* spgemm_numeric_to_host: spgemm_numeric (same preconditions, same device C)
 * that also copies C into host memory while the product is still being
 * computed.  The clusters are taken in nchunks consecutive ranges of cluster
 * ids (1..SGC_MAX_STREAM_CHUNKS; fewer when there are fewer clusters).  After
 * range g, every original row below the smallest row of the clusters of the
 * later ranges is final; those rows' C->col / C->val segments are copied to
 * host_col / host_val (nnz(C) elements each, at the same offsets as on the
 * device) on copy_stream while range g + 1 computes on stream.  host_row_ptr
 * (nrows + 1 elements) receives C->row_ptr when it is not NULL.  The overlap
 * is largest when clusters are ordered by their smallest row (as the
 * hcluster_reorder* calls order them); any order gives the same result.
 * Host buffers should be page-locked for the copies to run asynchronously.
 * nchunks = 0 selects the direct mode: the numeric kernels store C's entries
 * straight into host_col / host_val through their device-mapped addresses
 * (page-locked memory from cudaHostAlloc or cudaHostRegister, mapped for the
 * device; anything else is rejected with SGC_INVALID_ARG), so the transfer
 * overlaps the whole numeric phase whatever the cluster order; C->col and
 * C->val are not written and may be NULL.
 * copy_stream: a stream of the caller's other than stream (not NULL).
 * The range mode synchronises stream once, before the first range, to read
 * the range boundaries; the direct mode does not synchronise.  In both, on
 * return every copy is ordered before the work enqueued on stream afterwards,
 * so the host buffers are complete once stream is.  Errors: nchunks outside
 * 0..SGC_MAX_STREAM_CHUNKS, copy_stream NULL or equal to stream, NULL host
 * buffers with nnz(C) > 0, or (direct mode) host buffers the device cannot
 * address: SGC_INVALID_ARG; a workspace below spgemm_workspace_size:
 * SGC_WORKSPACE_TOO_SMALL.  Device-side failures are reported by
 * sgc_workspace_status. */
#define SGC_MAX_STREAM_CHUNKS 64
int spgemm_numeric_to_host(const sgc_csr_cluster* A, const sgc_csr* B, sgc_csr* C, int64_t* host_row_ptr,
                           int32_t* host_col, void* host_val, int32_t nchunks, void* ws, size_t ws_bytes,
                           const sgc_options* opt, void* stream, void* copy_stream);

/* ---------------------------------------------------------------------------
 * Plain row-wise Gustavson SpGEMM C = A * B with A in CSR (Sec. 2.2, Fig. 1):
 * the comparison method.  Same binning, hash accumulators, sort and copy-out
 * as the cluster-wise path, one row per warp, B rows read straight from
 * global memory.  Same contracts as spgemm_workspace_size / spgemm_symbolic /
 * spgemm_numeric.
 * ------------------------------------------------------------------------- */
int spgemm_rowwise_workspace_size(const sgc_csr* A, const sgc_csr* B, const sgc_options* opt,
                                  size_t* bytes);
int spgemm_rowwise_symbolic(const sgc_csr* A, const sgc_csr* B, int64_t* c_row_ptr,
                            int64_t* c_nnz_host, void* ws, size_t ws_bytes,
                            const sgc_options* opt, void* stream);
int spgemm_rowwise_numeric(const sgc_csr* A, const sgc_csr* B, sgc_csr* C, void* ws,
                           size_t ws_bytes, const sgc_options* opt, void* stream);

/* ---------------------------------------------------------------------------
 * Hierarchical clustering (Sec. 3.3, Algorithm 3, "Construct Hierarchical
 * Cluster"): candidate row pairs from SpGEMM_TopK(A, A^T) -- the structural
 * product A*A^T with all values 1 gives the overlap c_ij of rows i and j, the
 * Jaccard score is c_ij / (nnz_i + nnz_j - c_ij) -- then a max-heap of pairs
 * merged by union-find into clusters of at most max_cluster rows.
 *
 * hcluster_workspace_size: device workspace bytes for both calls below.
 *
 * hcluster_candidates: for every row i of A (any shape; only the pattern is
 * read), its `topk` best partners j != i with score > jacc_th, best first
 * (score compared exactly as integers; ties: smaller j first; the threshold
 * test is c > jacc_th * u in FP64): cand_j[i*topk + r] (-1 past the last),
 * cand_inter / cand_union the overlap and union sizes.  Device int32 arrays
 * of nrows*topk, caller-owned.  1 <= topk <= 31.  Asynchronous.
 *
 * hcluster_reorder: the clusters of Algorithm 3 with topk = max_cluster - 1
 * (1 <= max_cluster <= 32).  Readings where the paper is open: the merge loop
 * runs until the heap is empty; two roots merge only if the result has at
 * most max_cluster rows, the smaller row id becoming the root; when a popped
 * row is not a root, the pair of roots is scored and pushed if above the
 * threshold and never seen before; the heap orders by score, then smaller i,
 * then smaller j.  Output: perm (device int32, nrows: position -> row) and
 * cluster_ptr (device int64, capacity nrows+1): clusters ordered by their
 * smallest row, rows ascending within a cluster; *nclusters_host receives the
 * count.  The candidate search runs on the GPU; the heap and union-find run on
 * the host (A's pattern is copied to the host).  Synchronises.
 * ------------------------------------------------------------------------- */
int hcluster_workspace_size(const sgc_csr* A, int32_t max_cluster, size_t* bytes);

/* hcluster_reorder_parallel: a round-parallel variant of Algorithm 3's merge
 * (not in the paper), same candidate edges, same priority order, same
 * workspace and output conventions as hcluster_reorder.  Each round, every
 * candidate edge joining two clusters whose sizes sum to at most max_cluster
 * proposes to both; a cluster keeps its highest-priority proposal; edges kept
 * by both of their clusters merge them (the smaller root survives).  Rounds
 * run on the device until one merges nothing.  Scores are those of the
 * original row pairs (no re-scoring of root rows), so the clusters can differ
 * from hcluster_reorder's; C does not depend on the clustering.  Synchronises. */
int hcluster_reorder_parallel(const sgc_csr* A, float jacc_th, int32_t max_cluster, int32_t* perm,
                              int64_t* cluster_ptr, int64_t* nclusters_host, void* ws, size_t ws_bytes,
                              void* stream);

/* Cluster sources over A's own row order (Sec. 3.2), for comparison with
 * hierarchical clustering.  Both give perm = identity (position -> row),
 * cluster_ptr (device, int64, nclusters + 1 entries; at most nrows + 1) and
 * *nclusters_host.
 * cluster_fixed_length: clusters of K consecutive rows (1 <= K <= 32), the
 *   last one shorter.  Asynchronous.
 * cluster_variable_length: Algorithm 2.  A cluster's first row is its
 *   representative; the following row joins while Jaccard(representative,
 *   row) >= jacc_th (tested as inter >= jacc_th * union in FP64; an empty
 *   union ends the cluster) and the cluster has fewer than max_cluster rows
 *   (1..32).  The per-row run lengths are computed on the device; the chain of
 *   cluster starts is followed on the host.  Synchronises the stream. */
int cluster_fixed_length(int64_t nrows, int32_t K, int32_t* perm, int64_t* cluster_ptr, int64_t* nclusters_host,
                         void* stream);
int cluster_variable_length(const sgc_csr* A, float jacc_th, int32_t max_cluster, int32_t* perm,
                            int64_t* cluster_ptr, int64_t* nclusters_host, void* stream);
/* Cluster ordering by locality (the question of Sec. 4.3, whether a reordering
 * and the cluster-wise product compose, for the order in which clusters are
 * processed): reorders the clusters given by perm / cluster_ptr (device,
 * nrows and nclusters + 1 entries, as the hcluster_* calls return them) in
 * place so that clusters near each other in A's graph come close together,
 * for the B rows they share to hit in L2.  A must be square; its pattern is
 * the graph.  A breadth-first search on the device from row perm[0] gives
 * every row its distance (unique, so the result does not depend on timing);
 * a cluster's key is the smallest distance of its rows (rows not reached rank
 * last), and the clusters are sorted by key, ties in their previous order, on
 * the host.  Rows inside a cluster keep their order; C does not depend on the
 * order of clusters (build CSR_Cluster again after reordering).
 * *nlevels_host (nullable) receives the number of BFS levels.  ws: device
 * workspace of cluster_order_workspace_size(nrows, nclusters) bytes.
 * Synchronises (once per BFS level). */
int cluster_order_workspace_size(int64_t nrows, int64_t nclusters, size_t* bytes);
int cluster_order_bfs(const sgc_csr* A, int32_t* perm, int64_t* cluster_ptr, int64_t nclusters, int32_t* nlevels_host,
                      void* ws, size_t ws_bytes, void* stream);
int hcluster_candidates(const sgc_csr* A, float jacc_th, int32_t topk, int32_t* cand_j, int32_t* cand_inter,
                        int32_t* cand_union, void* ws, size_t ws_bytes, void* stream);
int hcluster_reorder(const sgc_csr* A, float jacc_th, int32_t max_cluster, int32_t* perm, int64_t* cluster_ptr,
                     int64_t* nclusters_host, void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Batched products and CUDA graphs (no counterpart in the paper, which
 * motivates repeated SpGEMMs with betweenness centrality, Sec. 4.2).
 *
 * csr_batch_pack: k independent products A_i * B_i are one product of the
 * block-diagonal matrices diag(A_i) * diag(B_i), whose result is diag(C_i);
 * this packs k CSR matrices (host array `mats` of structs holding device
 * pointers, one value type) into one block-diagonal CSR `out` whose arrays the
 * caller allocated with nrows = sum nrows_i, ncols = sum ncols_i, nnz = sum
 * nnz_i.  row_off / col_off (host, k+1 each) receive the block offsets: C_i is
 * rows [row_off[i], row_off[i+1]) of the packed C, its columns shifted by the
 * B blocks' column offsets.  Asynchronous (2k small launches + k copies).
 *
 * spgemm_graph_create: captures spgemm_symbolic (without the host read of
 * nnz) followed by spgemm_numeric into one CUDA graph on `stream` (a created
 * stream, not the legacy default stream) and instantiates it.  C must be
 * allocated with the nnz a previous spgemm_symbolic on the same structure
 * returned; the graph recomputes row pointer, columns and values on each
 * launch, so values of A and B may change between launches, the structure
 * may not.  All bins, grids and shared-memory classes are fixed at capture;
 * the persistent kernels read their work counts on the device.
 * spgemm_graph_launch / spgemm_graph_destroy: replay on a stream / free.
 * ------------------------------------------------------------------------- */
int csr_batch_pack(int32_t k, const sgc_csr* mats, sgc_csr* out, int64_t* row_off, int64_t* col_off,
                   void* stream);
typedef struct sgc_graph sgc_graph;
int spgemm_graph_create(const sgc_csr_cluster* A, const sgc_csr* B, sgc_csr* C, void* ws, size_t ws_bytes,
                        const sgc_options* opt, void* stream, sgc_graph** graph);
int spgemm_graph_launch(sgc_graph* graph, void* stream);
int spgemm_graph_destroy(sgc_graph* graph);

/* ---------------------------------------------------------------------------
 * Learned per-cluster output-column predictor and the symbolic-free path.
 * The paper has no predictor (its future work names learned choices, Sec. 5);
 * this library predicts, per cluster, n_out = the number of distinct output
 * columns of the cluster's rows (the cluster's nonzeros in CSR_Cluster form of
 * C) with an FP32 MLP 8 -> 32 -> 32 -> 1 (ReLU), target log1p(n_out).
 *
 * cluster_features: 8 FP32 features per cluster (row-major nclusters x 8):
 *   K/32, log1p(T)/8, log1p(nnz of the rows)/8, log1p(U)/8,
 *   log1p(sum of row flop bounds)/8, log1p(max row flop bound)/8,
 *   log1p(ncols(B))/16, (last - first union column + 1)/ncols(B);
 *   T = union columns, U = sum of nnz(B_t) over them, row flop bound
 *   ub_l = sum of nnz(B_t) over the row's columns.  Asynchronous.
 * nnz_predictor_targets: training targets from a completed spgemm_symbolic
 *   (ws: its workspace; c_row_ptr: C's row pointer it wrote): y[c] =
 *   log1p(n_out) for the clusters the symbolic phase handled in the cluster
 *   kernel and for one-row clusters (whose n_out is their row's count), -1 for
 *   the others (ignored by training); y_total[c] (nullable) = log1p(nnz_c),
 *   nnz_c = the summed counts of the cluster's rows (always known).
 * Parameters: 1377 FP32 values W1[32][8], b1[32], W2[32][32], b2[32], w3[32], b3.
 * nnz_predictor_train: `steps` Adam steps (beta 0.9/0.999, eps 1e-8, rate lr)
 *   from `init`, batch `batch` (a multiple of 32, at most
 *   SGC_NNZ_PREDICTOR_MAX_BATCH) samples order[s*batch .. +batch) at step s,
 *   loss = mean over valid samples (y >= 0) of (yhat - y)^2 / 2.  Data
 *   parallel: one CTA per 32 samples of the batch in one cooperative launch;
 *   each CTA sums its samples' gradients in sample order, and after a grid
 *   barrier every CTA adds the CTAs' sums in CTA order and applies the same
 *   update, so the result is deterministic.  loss_out: per step (nullable).
 *   ws: device workspace of nnz_predictor_train_workspace_size(batch) bytes;
 *   a grid barrier that does not complete within its bounded wait records
 *   SGC_DEVICE_TIMEOUT there (read it with sgc_workspace_status).
 *   Asynchronous.
 * nnz_predictor_grad: the loss and gradient of one batch (samples idx[0..batch)),
 *   same workspace rule.
 * nnz_predictor_infer: yhat for n samples.
 *
 * spgemm_learned_*: C = A*B without the exact symbolic pass.
 *   plan: features -> MLP (or the caller's per-cluster capacities) -> per
 *     cluster n_cap = min(min(U, ncols(B)), max(1, ceil(margin * scale *
 *     max(expm1(yhat), 0)))) (FP32), the capacity of the cluster's column
 *     table and accumulators; with params_total, nnz_hat_c = ceil(
 *     margin_total * scale * max(expm1(yhat_total), 0)), capped by the bound
 *     sum_l min(h_l, n_cap) (h_l = min(ub_l, ncols(B))), which is used instead
 *     when params_total is NULL.  The slab holds sum_c nnz_hat_c elements,
 *     returned in *slab_elems_host, split into 64 sub-pools: cluster c draws
 *     from sub-pool c mod 64, which holds the summed nnz_hat of its clusters.  Clusters of every size,
 *     one-row clusters included, are planned this way; a cluster whose
 *     working set exceeds shared memory goes to the exact path.  Synchronises.
 *   phase1: one cluster-wise pass computes every planned cluster whose n_out
 *     <= n_cap, counts its rows, reserves their total from its sub-pool with
 *     one atomic and writes the rows there (positions in the slab depend on
 *     timing, C does not); a cluster with more output columns than n_cap
 *     (an under-prediction), or one that finds its sub-pool exhausted, is
 *     flagged and its rows go through the exact symbolic pass; c_row_ptr
 *     (nrows+1) is C's row pointer; *c_nnz_host = nnz(C), *n_overflow_host =
 *     clusters sent to the exact path.  Synchronises.
 *   phase2: copies slab rows into C and runs the exact numeric pass on the
 *     flagged clusters.  C (allocated by the caller with nnz(C)) equals the
 *     result of spgemm_symbolic + spgemm_numeric exactly.  C->col and C->val
 *     may be device memory or page-locked host memory mapped for the device
 *     (cudaHostAlloc / cudaHostRegister): the kernels then store C's entries
 *     straight into host memory; pageable host memory is rejected with
 *     SGC_INVALID_ARG.  Asynchronous.
 *   All three take the same workspace (spgemm_learned_workspace_size).
 * ------------------------------------------------------------------------- */
#define SGC_NNZ_PREDICTOR_PARAMS 1377
#define SGC_NNZ_PREDICTOR_MAX_SETS 2

/* nnz_predictor_save / nnz_predictor_load: checkpoints of trained predictors.
 * A file holds nsets (1..SGC_NNZ_PREDICTOR_MAX_SETS) parameter sets of
 * SGC_NNZ_PREDICTOR_PARAMS FP32 values each, back to back in `params` (device),
 * and a metadata string: magic "SGCNNZP2", uint32 nsets, uint32 metadata
 * length, the metadata bytes, the parameters; little-endian.  Files written
 * with magic "SGCNNZP1" (one set) load as one set.
 * save: meta may be NULL.  Synchronises the stream (reads params), then writes
 *   the file; SGC_INVALID_ARG if the file cannot be opened, SGC_CUDA_ERROR if
 *   a write fails.
 * load: writes *nsets_out sets into params (device, room for max_sets sets)
 *   and, when meta is not NULL, up to meta_cap - 1 metadata bytes and a
 *   terminating 0.  SGC_INVALID_ARG for a missing file, a wrong magic, size or
 *   set count, or more sets than max_sets.  Synchronises. */
int nnz_predictor_save(const char* path, const float* params, int32_t nsets, const char* meta, void* stream);
int nnz_predictor_load(const char* path, float* params, int32_t max_sets, int32_t* nsets_out, char* meta,
                       size_t meta_cap, void* stream);
typedef struct sgc_predictor {
  const float* params;        /* device, SGC_NNZ_PREDICTOR_PARAMS FP32 values: predicts log1p(n_out)
                                 (ignored if ncap is set) */
  float margin;               /* capacity margin over the prediction (e.g. 1.25) */
  float scale;                /* multiplies both predictions (1 = as predicted) */
  const int32_t* ncap;        /* optional device array of nclusters capacities used instead of the MLP */
  const float* params_total;  /* optional device parameter set predicting log1p(nnz_c), the cluster's
                                 output nonzeros (its rows' counts summed), which sizes the slab; NULL:
                                 the slab is sized by the bound sum_l min(h_l, n_cap) */
  float margin_total;         /* margin of the slab over the summed nnz_c predictions; 0 = margin */
  int32_t reserved;
} sgc_predictor;

int cluster_features(const sgc_csr_cluster* A, const sgc_csr* B, float* features, void* stream);
int nnz_predictor_targets(const sgc_csr_cluster* A, const sgc_csr* B, const void* ws, size_t ws_bytes,
                          const int64_t* c_row_ptr, float* y, float* y_total, void* stream);
int nnz_predictor_infer(const float* params, const float* features, int64_t n, float* yhat, void* stream);
#define SGC_NNZ_PREDICTOR_MAX_BATCH 4096
int nnz_predictor_train_workspace_size(int32_t batch, size_t* bytes);
int nnz_predictor_grad(const float* params, const float* features, const float* y, const int32_t* idx,
                       int32_t batch, float* grad, float* loss, void* ws, size_t ws_bytes, void* stream);
int nnz_predictor_train(const float* features, const float* y, int64_t n, const int32_t* order, int64_t steps,
                        int32_t batch, float lr, const float* init, float* params_out, float* loss_out, void* ws,
                        size_t ws_bytes, void* stream);
int spgemm_learned_workspace_size(const sgc_csr_cluster* A, const sgc_csr* B, const sgc_options* opt,
                                  size_t* bytes);
int spgemm_learned_plan(const sgc_csr_cluster* A, const sgc_csr* B, const sgc_predictor* pred,
                        int64_t* slab_elems_host, void* ws, size_t ws_bytes, const sgc_options* opt, void* stream);
int spgemm_learned_phase1(const sgc_csr_cluster* A, const sgc_csr* B, int32_t* slab_col, void* slab_val,
                          int64_t* c_row_ptr, int64_t* c_nnz_host, int64_t* n_overflow_host, void* ws,
                          size_t ws_bytes, const sgc_options* opt, void* stream);
int spgemm_learned_phase2(const sgc_csr_cluster* A, const sgc_csr* B, const int32_t* slab_col,
                          const void* slab_val, sgc_csr* C, void* ws, size_t ws_bytes, const sgc_options* opt,
                          void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SGC_H_ */
