/*
 * msf.h -- C ABI of the GB300 minimum spanning forest library.
 *
 * The library computes the minimum spanning forest (MSF) of undirected
 * weighted graphs with the algebraic Awerbuch-Shiloach method of Baer,
 * Kanakagiri and Solomonik, "Parallel Minimum Spanning Forest Computation
 * using Sparse Matrix Kernels" (arXiv:2110.04865):
 *   - Sec. 3.1 / Algorithm 2 (multilinear and projection steps): the kernel
 *     q_i = MinWeight_j f(p_i, a_ij, p_j) and its projection r_{p_i} = min q_i;
 *   - Algorithm 2 (hooking and tie breaking): star hooking, 2-cycle removal;
 *   - Sec. 4.2 / Algorithm 3: complete shortcutting of every tree to a star;
 *   - Algorithm 2 (loop test): repeat until no star hooks.
 * All of it runs as CUDA kernels on one GPU (sm_103a).
 *
 * Conventions shared by every call
 *   * Graphs are undirected.  Vertices are 0 .. n-1.  Edge e of the input
 *     list (src[e], dst[e], w[e]) is an undirected edge; self-loops are
 *     accepted and never part of the forest; parallel edges are separate.
 *   * Weights are float32 (MSF_F32) or uint32 (MSF_U32), passed as `const
 *     void*`.  The paper assumes distinct weights (Sec. 2); here edges are
 *     ordered strictly by (weight, input index), which makes the forest
 *     unique.  For float32, -0 == +0, +-inf are allowed, NaN is rejected.
 *   * Pointers may be device pointers or host pointers; the library looks
 *     them up (cudaPointerGetAttributes).  Host inputs are copied to the
 *     device inside the call; host outputs are written back before the call
 *     returns.  Caller buffers are only read or written during the call.
 *   * `stream` is a cudaStream_t (NULL = the legacy default stream).  All
 *     work is ordered on it; the calls that return results synchronize it.
 *   * Every call returns an msf_status; on failure msf_last_error() gives a
 *     message (thread-local, valid until the next call on that thread) and
 *     the outputs are undefined.
 */
#ifndef MSF_H
#define MSF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct msf_graph msf_graph; /* opaque; owns the device CSR */

enum msf_wtype { MSF_F32 = 0, MSF_U32 = 1 };

enum msf_status {
  MSF_OK = 0,
  MSF_ERR_INVALID_ARG = 1,    /* bad size, index out of [0,n), NaN weight, bad offsets */
  MSF_ERR_OOM = 2,            /* device or host allocation failed */
  MSF_ERR_CUDA = 3,           /* a CUDA runtime call failed */
  MSF_ERR_ROUND_LIMIT = 4,    /* more rounds than the limit (default 64) */
  MSF_ERR_SHORTCUT_LIMIT = 5, /* shortcutting did not settle (default 64 passes) */
  MSF_ERR_TOO_LARGE = 6,      /* n >= 2^31 or m >= 2^32 - 1 */
  MSF_ERR_CHECK = 7           /* an internal consistency check failed on the device */
};

/*
 * msf_build_csr -- store a graph on the device as a symmetric CSR.
 *
 * The adjacency matrix A of Sec. 2 (a_ij = w(i,j), absent entries infinite,
 * as in Algorithm 2) is kept as a doubly compressed CSR over the vertices of
 * nonzero degree.  Each slot holds the column j and the 64-bit key
 * ord(w) * 2^32 + e, where e is the undirected edge id; both directions of an
 * edge carry the same key.
 *
 *   n        number of vertices, 0 <= n < 2^31.
 *   m        COO form: number of edges, 0 <= m < 2^32 - 1.
 *            CSR form: number of slots row_ptr[n].
 *   src,dst  COO form (row_ptr == NULL): int32[m] endpoints in [0, n).
 *   row_ptr  CSR form: int64[n+1]; dst is then the column array int32[m]
 *            and src is ignored.  Only slots with row < column are read: slot
 *            s with row i < dst[s] is the undirected edge with id s.  Slots
 *            with row >= column are ignored (a symmetric matrix repeats each
 *            edge there), and their mask entries stay 0.
 *   w        weights, float32 or uint32, [m] (per slot in CSR form).
 *   wtype    MSF_F32 or MSF_U32.
 *   flags    must be 0 (reserved).
 *   out      receives the handle; release it with msf_free.
 * Validation runs on the device before the CSR is written; the call
 * synchronizes `stream` and returns MSF_ERR_INVALID_ARG on a bad index or a
 * NaN weight.
 */
int msf_build_csr(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                  const int64_t *row_ptr, const void *w, int wtype, uint32_t flags,
                  void *stream, msf_graph **out);

/*
 * msf_compute -- minimum spanning forest of a built graph (Algorithm 2 with
 * complete shortcutting, Sec. 4.2).  The round loop runs on the device as a
 * CUDA graph with a conditional while node; the host waits once at the end.
 *
 *   edge_mask  uint8[m]: 1 for forest edges, 0 otherwise (indexed like the
 *              input edges, or like the slots in CSR form).
 *   labels     int32[n]: smallest vertex id of each vertex's component.
 *   total      double[1]: exact sum of the forest weights rounded once to
 *              double (float32: a long accumulator over all exponents; +inf
 *              if an infinite weight is in the forest).
 * Any output may be NULL.  Synchronizes `stream`.  The graph can be computed
 * any number of times.  When the round limit ends the loop
 * (MSF_ERR_ROUND_LIMIT), edge_mask and total describe the forest edges found
 * in the completed rounds and, with complete shortcutting, labels the trees
 * after them; other errors leave the outputs undefined.
 */
int msf_compute(msf_graph *g, uint8_t *edge_mask, int32_t *labels, double *total, void *stream);

/*
 * msf_compute_batched -- forests of G independent graphs in one call.
 *
 * The graphs are stored as one disjoint union and solved by one launch of the
 * same round loop; results are split per graph.
 *   voff, eoff  HOST int64[G+1] vertex and edge offsets, voff[0] = eoff[0] = 0,
 *               non-decreasing.
 *   src, dst    int32[eoff[G]] endpoints in LOCAL ids: for e in graph g,
 *               0 <= src[e] < voff[g+1] - voff[g].
 *   w           float32 or uint32 [eoff[G]].
 *   edge_mask   uint8[eoff[G]];  labels int32[voff[G]] (LOCAL ids);
 *   totals      double[G].
 * Synchronizes `stream`.
 */
int msf_compute_batched(int32_t G, const int64_t *voff, const int64_t *eoff, const int32_t *src,
                        const int32_t *dst, const void *w, int wtype, uint8_t *edge_mask,
                        int32_t *labels, double *totals, void *stream);

/* msf_free -- release a graph and its device memory (NULL is ignored).  The
 * memory returns to the library's caching allocator. */
void msf_free(msf_graph *g);

/* msf_last_error -- message of the last failed call on this thread. */
const char *msf_last_error(void);

/*
 * msf_min_edge -- one application of the multilinear kernel and its
 * projection (Sec. 3.1; the multilinear and projection steps of Algorithm 2):
 *   r_k = min { key(i,j) : p_i = k, p_i != p_j }   for every vertex k,
 * with key(i,j) = ord(w) * 2^32 + edge id and UINT64_MAX for "no edge".
 *   parent  int32[n], a star forest: every parent[i] is a root
 *           (parent[parent[i]] == parent[i]); under complete shortcutting
 *           every vertex lies in a star, so f needs no star test.
 *   r       uint64[n] output.
 * Runs on the graph's original CSR.  Synchronizes `stream`.
 */
int msf_min_edge(msf_graph *g, const int32_t *parent, uint64_t *r, void *stream);

/*
 * msf_min_edge_part -- msf_min_edge restricted to one part of a 1-D
 * partition of the CSR (the single-node counterpart of Sec. 4.1's
 * distribution of A over processes): the graph's nnz directed slots, in row
 * order, are cut into `nparts` contiguous ranges at multiples of 512 slots,
 *   part k: [512 * floor(k * nnz / (512 * nparts)), the same for k + 1),
 * the last part ending at nnz; a row that crosses a cut contributes to both
 * parts.  r receives the projection of part `part` alone:
 *   r_k = min { key(i,j) : slot (i,j) in the part, p_i = k, p_i != p_j },
 * UINT64_MAX where the part has none.  The elementwise minimum of the nparts
 * partial projections (for instance a MIN all-reduce across the processes
 * that own the parts) is msf_min_edge's r.
 *   parent  int32[n] star forest; r uint64[n] output (device or host memory).
 *   0 <= part < nparts; nparts >= 1.
 * Synchronizes `stream`.
 */
int msf_min_edge_part(msf_graph *g, const int32_t *parent, int32_t part, int32_t nparts, uint64_t *r,
                      void *stream);

/*
 * msf_apply_round -- the rest of one round of Algorithm 2 from a projection
 * computed elsewhere (the elementwise minimum of msf_min_edge_part's partial
 * projections over all parts): hooking (every root k with r_k != UINT64_MAX
 * hooks along edge id(r_k) onto the parent of its far endpoint), tie
 * breaking of the 2-cycles (the smaller root stays a root) with the forest
 * edges marked in edge_mask, then complete shortcutting (Sec. 4.2, Algorithm
 * 3), so that parent is again a star forest.  Every process holding the same
 * parent and r computes the same result, so the chase of the changed parents
 * needs no all-gather.
 *   r          uint64[n] DEVICE memory, the reduced projection; on return every
 *              entry is UINT64_MAX (ready for the next round's reduction).
 *   parent     int32[n] DEVICE memory, star forest, updated in place (start
 *              from parent[i] = i).
 *   edge_mask  uint8[m] DEVICE memory: the call sets edge_mask[e] = 1 for the
 *              forest edges found in this round and writes nothing else
 *              (start from zeros).
 *   labels     int32[n] DEVICE memory or NULL: when given, the smallest vertex
 *              id of each vertex's tree after the round (after the last round:
 *              msf_compute's labels).
 *   hooks      HOST int64: the number of roots that hooked (forest edges
 *              added); 0 means the forest is complete.
 * Errors: MSF_ERR_CHECK when a key of r does not leave its star (r is not a
 * projection of this graph for this parent); MSF_ERR_SHORTCUT_LIMIT as in
 * msf_compute.  Synchronizes `stream`.
 */
int msf_apply_round(msf_graph *g, uint64_t *r, int32_t *parent, uint8_t *edge_mask, int32_t *labels,
                    int64_t *hooks, void *stream);

/*
 * msf_connected_components -- connected components of a built graph by the
 * Awerbuch-Shiloach connectivity algorithm in its linear-algebra form
 * (Sec. 2.4): each round every star vertex takes the smallest parent among
 * its neighbours, p^h_i; conditional hooking hooks the star root onto p^h_i
 * when p^h_i < p_i; after a starcheck, the vertices still in stars repeat it
 * without the check over the neighbours whose trees are not stars
 * (unconditional hooking: a non-star tree does not move in this step, so no
 * cycle forms);
 * then shortcutting makes every tree a star.  Stops after a round without a
 * hook.  Edge weights play no part.
 *   labels  int32[n]: smallest vertex id of each vertex's component (the same
 *           labels msf_compute returns).
 * Synchronizes `stream`.
 */
int msf_connected_components(msf_graph *g, int32_t *labels, void *stream);

/*
 * msf_weight_backward -- gradient of the forest weight(s) with respect to the
 * edge weights: grad_w[e] = edge_mask[e] ? (float)grad_total[graph(e)] : 0.
 * Where weights are distinct the forest is locally constant, so the
 * derivative of sum_{e in F} w_e is the membership indicator.
 *   m           number of edges.
 *   G, eoff     G >= 1 graphs; eoff HOST int64[G+1] (may be NULL when G == 1).
 *   edge_mask   uint8[m]; grad_total double[G]; grad_w float32[m].
 * Does not synchronize `stream` when every pointer is a device pointer.
 */
int msf_weight_backward(int64_t m, int32_t G, const int64_t *eoff, const uint8_t *edge_mask,
                        const double *grad_total, float *grad_w, void *stream);

/*
 * msf_forest_weight_noalloc -- exact forest weight per graph without any
 * device allocation.  The paper has no counterpart: this is a service entry
 * point for callers that cannot allocate device memory at call time -- for
 * example code running under another allocator that owns the device memory
 * budget, plug-ins whose host application forbids cudaMalloc/cudaFree, or
 * latency-bound loops that cannot pay for the device synchronisation that
 * cudaMalloc and cudaFree imply.
 *
 *   totals[g] = exact sum of w[e] over e in graph g with edge_mask[e] == 1,
 *               rounded once to double (float32: long accumulator over all
 *               exponents, +inf if an infinite weight is selected, NaN if a
 *               NaN weight is selected or both infinities are; uint32:
 *               64-bit integer sum), the same value msf_compute(_batched)
 *               returns for its own mask.
 *   G          1 <= G <= 1024 graphs; larger G returns MSF_ERR_TOO_LARGE.
 *   m          number of edges (all graphs).
 *   eoff       HOST int64[G+1] edge offsets (eoff[0] = 0, eoff[G] = m); may be
 *              NULL when G == 1.
 *   edge_mask  uint8[m], w (float32 or uint32)[m], totals double[G]: DEVICE
 *              memory only (host buffers would need staging memory and are
 *              rejected with MSF_ERR_INVALID_ARG).
 * Scratch: a fixed 2 MiB + 12 KiB array in the library's device image (256
 * 64-bit accumulators per graph, the copied offsets and a NaN flag per
 * graph), present on every GPU that loads the library until the process
 * exits.  The accumulators and flags are cleared at the start of every call,
 * and every call shares the one array: calls whose work overlaps on a GPU
 * (different streams, or host threads without ordering) race and give wrong
 * totals.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it for the life of the device's primary
 * context; make that first call before any stream capture, and do not call
 * the library on a device again after cudaDeviceReset.  The call is
 * asynchronous: totals are ready when `stream` reaches this point.  It calls
 * no cudaMalloc, cudaFree or allocating routine.
 */
int msf_forest_weight_noalloc(int32_t G, int64_t m, const int64_t *eoff, const uint8_t *edge_mask,
                              const void *w, int wtype, double *totals, void *stream);

/* Statistics of the last msf_compute on a graph. */
typedef struct msf_stats {
  int64_t n, m;          /* vertices and edges */
  int64_t nnz;           /* directed CSR slots of the original graph */
  int64_t rows;          /* CSR rows (vertices of nonzero degree) */
  int32_t rounds;        /* rounds of the loop, the final one without hooks included */
  int32_t compactions;   /* rounds that compacted the edge list */
  int64_t forest_edges;  /* edges in the forest */
  int32_t jump_steps;    /* pointer-jumping steps over all rounds */
  float min_edge_ms;     /* duration of the sweep kernel in the last msf_min_edge call
                            (CUDA events on the caller's stream around that launch only) */
  int32_t cc_rounds;     /* rounds of the last msf_connected_components call */
  int32_t kernels;       /* kernels the library ran for msf_build_csr plus the last msf_compute
                            (host launches and the executed nodes of the round-loop graph) */
  int32_t builder;       /* the CSR builder msf_build_csr ran: 1 per-vertex atomic, 2 radix,
                            3 bucketed (MSF_OPT_BUILD's numbering) */
} msf_stats;

int msf_get_stats(const msf_graph *g, msf_stats *out);

/* Tuning options (process-wide). */
enum msf_option {
  MSF_OPT_COMPACT_TAU = 0,   /* compact when live slots < tau * slots (0 < tau < 1; default 0.5; 0 = never) */
  MSF_OPT_ROUND_LIMIT = 1,   /* maximum rounds (default 64) */
  MSF_OPT_JUMP_LIMIT = 2,    /* maximum shortcut passes per round (default 64) */
  MSF_OPT_SLOTS_PER_LANE = 3,/* min-edge tile: slots per lane, 4, 8 or 16 (default 4) */
  MSF_OPT_BLOCKS_PER_SM = 4, /* min-edge grid: resident blocks per SM (1..8, default 4) */
  MSF_OPT_PREFETCH = 5,      /* min-edge sweep loads the next tile early: 0 or 1 (default 0) */
  MSF_OPT_EXEC_MODE = 6,     /* 0 = device round loop in a CUDA graph (default); 1 = host-driven
                                loop, one launch per kernel and a host wait per decision (for
                                profiling kernels individually) */
  MSF_OPT_SHORTCUT = 7,      /* shortcut schedule, one of msf_shortcut (default MSF_SHORTCUT_CSP) */
  MSF_OPT_OS_THRESHOLD = 8,  /* MSF_SHORTCUT_OPTIMIZED: chase the changed roots when at most this
                                many roots hooked in the round, else full passes (default 1310720) */
  MSF_OPT_KERNEL = 9,        /* 0 = fused multilinear min-edge kernel (default); 1 = pairwise
                                formulation of Sec. 4.1: one pass writes p_j next to every slot
                                (nnz extra writes and an nnz-word buffer), a second reduces */
  MSF_OPT_BUILD = 10,        /* CSR builder: 0 = automatic (default: bucketed from 2^20 edges
                                unless a sample shows locality -- consecutive sampled edges with
                                endpoints close together, as in a lattice listed vertex by vertex
                                or a batch listed graph by graph -- then per-vertex atomic
                                counters, as for small graphs), 1 = atomic,
                                2 = radix grouping, 3 = bucketed (rows grouped in at most 1024
                                buckets of consecutive vertices, counted in shared memory).  All
                                give the same CSR up to the order of slots inside a row. */
  MSF_OPT_EARLY_STOP = 11,   /* 1 (default): with complete shortcutting, end the loop after a
                                round that left at most one tree with an outgoing edge, instead
                                of running one more round that finds no hook; 0: always confirm */
  MSF_OPT_SWEEP = 12,        /* form of the multilinear min-edge sweep: 0 = tiles loaded into
                                registers by every lane (default); 1 = per-warp shared-memory
                                pipeline (bulk copies of columns and keys two tiles ahead, p_j
                                gathered by asynchronous copies one tile ahead); 2 = register
                                tiles loaded two ahead, p_j and row parents gathered one ahead
                                into shared memory.  Same results. */
  MSF_OPT_HOST_INPUT = 13,   /* edge arrays in host memory: 0 = copied to the device before the
                                build (default); 1 = page-locked host arrays are read in place by
                                the build kernels over the CPU-GPU link (pageable ones are still
                                copied).  Same results. */
  MSF_OPT_RELABEL = 14       /* 1 (default): the second round's min-edge sweep also writes every
                                slot's column as its current root into a copy of the column
                                array, which the later rounds read, so that their p_j gathers
                                touch only the roots left after the first round (4 bytes per slot
                                of device memory); 0: off.  Same results. */
};

/* Shortcut schedules (Sec. 2.3, Sec. 4.2, Sec. 7.1).  All give the same
 * forest, labels and total; they differ in rounds and work per round. */
enum msf_shortcut {
  MSF_SHORTCUT_CSP = 0,       /* complete shortcutting, Algorithm 3: the roots that hooked this
                                 round follow their parent chains to the final roots (passes of up
                                 to 16 hops each), then one gather for every vertex */
  MSF_SHORTCUT_ORIGINAL = 1,  /* original schedule (Algorithm 1): starcheck before hooking and
                                 before shortcutting, one shortcut step per round */
  MSF_SHORTCUT_FULL = 2,      /* complete shortcutting by full passes: every vertex takes its
                                 grandparent until no parent moves (the baseline of Sec. 4.2) */
  MSF_SHORTCUT_OPTIMIZED = 3  /* per round: CSP when at most MSF_OPT_OS_THRESHOLD roots hooked,
                                 else full passes (the optimized shortcut of Sec. 7.1) */
};
int msf_set_option(int option, double value);
double msf_get_option(int option);

#ifdef __cplusplus
}
#endif

#endif /* MSF_H */
