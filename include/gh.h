/*
 * gh.h -- C ABI of the GB300 grid-hopping polygonizer.
 *
 * The library turns a signed distance bound (SDB) into a triangle mesh with
 * the grid-hopping method of Markus & Suznjevic, "Theoretical and Empirical
 * Analysis of a Fast Algorithm for Extracting Polygons from Signed Distance
 * Bounds" (Sec. 3, Algorithm 1): N^2 rays are cast along +z through the cell
 * centres of an N^3 grid (Eq. 1-2); each ray evaluates the bound d = |f| at a
 * cell centre and jumps floor(d / h) cells ahead (the sphere-tracing
 * iteration of Eq. 3 on the cell lattice); a cell whose centre is within the
 * polygonization distance tau of the surface (Eq. 4) is marked, and only
 * marked cells get Marching Cubes.  The result equals Marching Cubes over all
 * N^3 cells (Sec. 5: all methods produce the same mesh).
 *
 * Every compute step runs in sm_103a CUDA kernels on the caller's stream; no
 * entry point has a CPU fallback.  All pointers named "device" must be
 * device memory of the current CUDA device.  Unless stated otherwise an
 * entry point returns GH_OK or one of the GH_ERR_* codes below and leaves a
 * readable message in gh_last_error().
 *
 * Conventions (the paper's unit cube generalised to a cube [lo, hi]^3):
 *   h = (hi - lo) / N; cell (i,j,k) = [lo + i h, lo + (i+1) h] x ...;
 *   cell id = (i*N + j)*N + k; lattice vertex (a,b,c) = lo + (a,b,c) h;
 *   inside <=> f < 0 (f == 0 counts as outside);
 *   Marching Cubes case = sum_b [f(corner b) < 0] << b with corner b at offset
 *   (b&1, b>>1&1, b>>2&1);
 *   the vertex on a crossing edge from lower endpoint A to upper endpoint B
 *   sits at t = fA / (fA - fB) from A;
 *   edge key = axis*(N+1)^3 + a + (N+1)*(b + (N+1)*c) with (a,b,c) the
 *   lattice coordinates of A -- equal keys denote the same mesh vertex;
 *   triangles are oriented so that (v1 - v0) x (v2 - v0) points towards f > 0.
 */
#ifndef GH_H_
#define GH_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define GH_OK 0
#define GH_ERR_ARG 1           /* invalid argument; nothing was enqueued        */
#define GH_ERR_CAPACITY 2      /* an output buffer was too small (see gh_mesh)  */
#define GH_ERR_CUDA 3          /* a CUDA call failed; message has the details   */
#define GH_ERR_NONFINITE 4     /* the SDB produced NaN or inf                   */
#define GH_ERR_UNIMPLEMENTED 5 /* combination not supported by the library        */
#define GH_ERR_DEVICE 6        /* the GPU is not an sm_103 device               */

/* ---- SDB kinds and their blob formats ---------------------------------- */
#define GH_SDB_CSG 0
#define GH_SDB_MLP 1

/* CSG blob: gh_csg_header followed by n_prim gh_csg_prim records.
 * f = op_{n-1}( ... op_1(d_0, d_1) ..., d_{n-1}) -- a left fold where union is
 * min (Sec. 4.3), subtract is max(f, -d) and intersect is max(f, d).  Every
 * primitive is an exact Euclidean distance, so f is a signed distance bound
 * (Sec. 1).  q = rot * (p - centre) is the point in the primitive's frame;
 * rot must be a rotation (|rot rot^T - I| <= 1e-4 entrywise, else
 * gh_create_sdb returns GH_ERR_ARG), and spheres do not read it.  The
 * evaluator skips a primitive whose distance provably cannot change the fold
 * (bounding-ball test, exact: the result equals the full fold bit for bit);
 * that test is only taken for positive sizes and |rot rot^T - I| <= 1e-6. */
#define GH_PRIM_SPHERE 0 /* param[0] = radius                                 */
#define GH_PRIM_TORUS 1  /* around local y: param[0] = major R, param[1] = r   */
#define GH_PRIM_BOX 2    /* exact box distance (Sec. 4.2), half sizes param[] */
/* 3..6 with the sphere, box and torus are the seven basic primitives of the
 * first test scene (Sec. 5.1); each is an exact distance, param[2] unused.
 * gh_backward differentiates all seven (centre and param[0..1]). */
#define GH_PRIM_CAPSULE 3  /* segment (0,-H,0)-(0,H,0) widened by r: param = H, r  */
#define GH_PRIM_CYLINDER 4 /* capped, around local y: param = radius r, half height H */
#define GH_PRIM_HEXPRISM 5 /* regular hexagon of apothem a in the local xz-plane   */
                           /* (edges facing 0, 60, ... degrees), |y| <= H: a, H   */
#define GH_PRIM_CONE 6     /* solid cone: base disc radius R at y = -H, apex at +H; */
                           /* R > 0 and H > 0 (else GH_ERR_ARG)                  */
#define GH_OP_UNION 0
#define GH_OP_SUBTRACT 1
#define GH_OP_INTERSECT 2
#define GH_MAX_PRIMS 256
typedef struct {
    int32_t n_prim;
    int32_t reserved[3];
} gh_csg_header;
typedef struct {
    int32_t type, op;
    float centre[3];
    float param[3];
    float rot[9]; /* row-major, world offset -> local frame */
    float pad[3];  /* ignored (the library's copy keeps derived data there) */
} gh_csg_prim; /* 80 bytes */

/* MLP blob (the neural SDB of Sec. 5.2, Eq. 7): gh_mlp_header followed by
 * float32 parameters packed as W0[width][3] b0[width] then n_mid times
 * { W[width][width] b[width] } then w_out[width] b_out[1] (row-major,
 * out x in, like torch.nn.Linear).  g = w_out . relu(W_mid ... relu(W0 p + b0)
 * ...) + b_out and f(p) = (|p| - r0 + alpha g(p)) / beta / lipschitz_scale.
 * flags = GH_MLP_NO_RADIAL drops the |p| term: f = (alpha g - r0) / beta /
 * lipschitz_scale, the form of the paper's own networks (SDB = network /
 * lambda, Sec. 5.2; alpha = beta = 1, r0 = 0).  A network trained with batch
 * normalisation is passed with the normalisation folded into the preceding
 * layer.  width must be 64, 128 or 256. */
typedef struct {
    int32_t width, n_mid;
    int32_t flags;
    int32_t reserved;
    float r0, alpha, beta, reserved_f;
} gh_mlp_header;
#define GH_MLP_NO_RADIAL 1

typedef struct gh_sdb gh_sdb; /* opaque; owned by the library */

typedef struct {
    int32_t kind;          /* GH_SDB_CSG | GH_SDB_MLP                          */
    const void *blob;      /* host pointer; copied, the caller keeps ownership */
    size_t blob_bytes;
    float lipschitz_scale; /* lambda >= 1 of Sec. 5.2; f is divided by it; 0 = 1 */
} gh_sdb_desc;

typedef struct {
    int32_t N;    /* cells per axis, 2 <= N <= 2048                          */
    float lo[3];  /* the polygonization volume; hi - lo must be equal on all */
    float hi[3];  /* three axes (a cube, Sec. 2)                            */
} gh_grid;

#define GH_FP32 0        /* every evaluation in FP32                           */
#define GH_BF16_REFINE 1 /* neural SDB: hop in BF16 with an error bound eps,   */
                         /* corners of candidate cells re-evaluated in FP32    */
/* GH_BF16_REFINE_X6: as GH_BF16_REFINE, but the corners are re-evaluated on
 * the tensor cores with split-BF16 products instead of FP32 FMAs: every FP32
 * operand of a hidden layer is split exactly into three BF16 parts and the
 * six part products of size >= 2^-16 of the product are accumulated in FP32
 * (the dropped three are below about 2^-23 of it).  Not FP32 arithmetic:
 * its error against exact arithmetic is of FP32's size, not bit-identical to
 * GH_FP32.  gh_eval takes it too (points evaluated that way). */
#define GH_BF16_REFINE_X6 2
/* The BF16 modes support widths 64, 128 and 256 with at most 8 hidden layers
 * (n_mid), 7 at width 256, and the split-BF16 evaluator at most 8; other
 * networks get GH_ERR_UNIMPLEMENTED for them (GH_FP32 takes any depth). */
#define GH_TAU_DIAGONAL 0      /* tau = sqrt(3) h: one cell diagonal (default) */
#define GH_TAU_HALF_DIAGONAL 1 /* tau = sqrt(3) h / 2: the tightest safe value */

typedef struct {
    int32_t precision; /* GH_FP32 | GH_BF16_REFINE | GH_BF16_REFINE_X6       */
                       /* (the two BF16 modes: neural SDBs only)             */
    int32_t tau_mode;  /* GH_TAU_*                                            */
    float eps;         /* BF16 bound |f_bf16 - f_fp32| <= eps/2; < 0 = the    */
                       /* SDB's calibrated value (gh_sdb_calibrate)           */
    int32_t sync;      /* 1: wait for the stream before returning, grow       */
                       /* internal scratch and retry when it overflowed, and  */
                       /* return device-side errors; 0: fully asynchronous,   */
                       /* errors land in stats->status                        */
    int32_t ray_block; /* tuning: threads per CTA of the analytic hopper      */
                       /* (128, 256 or 512; 0 = 256)                          */
    int32_t mlp_tiles; /* tuning: 128-row tiles per CTA of the BF16 engine    */
                       /* (1 or 2; 0 = 2)                                     */
    int32_t method;    /* GH_METHOD_HOP (Algorithm 1, default) or             */
                       /* GH_METHOD_ENUM: f at all (N+1)^3 lattice points and */
                       /* Marching Cubes on all N^3 cells (Sec. 2), FP32 only */
} gh_options;
#define GH_METHOD_HOP 0
#define GH_METHOD_ENUM 1

/* Counters written by the device (all int64 so a caller may read the struct
 * with one copy). */
typedef struct {
    int64_t status;          /* GH_OK or a GH_ERR_* code from the device      */
    int64_t columns;         /* N^2                                           */
    int64_t hop_evals;       /* f evaluations made by the rays                */
    int64_t marked_cells;    /* cells within tau                              */
    int64_t unique_vertices; /* lattice vertices evaluated for Marching Cubes:
                                the corners of marked cells except those whose
                                hop value |f| - eps exceeds sqrt(3)/2 h + eps
                                (plus a rounding margin), which hold no zero */
    int64_t refined_vertices;/* of those, re-evaluated in FP32 (BF16 path)    */
    int64_t surface_cells;   /* marked cells with 0 < case < 255              */
    int64_t triangles;       /* triangles produced (may exceed capacity)      */
    int64_t row_slots;       /* neural hopper: rows run, live or idle (a tile */
                             /* of 128 rows per step); hop_evals / row_slots  */
                             /* is the share of the GEMM rows doing work      */
    int64_t mesh_vertices;   /* crossing lattice edges = vertices of the      */
                             /* indexed mesh (when it is requested)           */
    int64_t reserved[6];
} gh_stats;

/* Output description; every buffer is caller-owned device memory.
 * tri_xyz:   [capacity_tris][3][3] float32 vertex positions (triangle soup).
 * tri_keys:  [capacity_tris][3] uint64 edge keys, or NULL.
 * n_tris:    one int64 written with the number of triangles produced.  When
 *            it exceeds capacity_tris only the first capacity_tris are written
 *            (in an unspecified order) and the call reports GH_ERR_CAPACITY.
 * cell_ids / cell_cases / capacity_cells / n_cells: optional (NULL) list of
 *            the surface cells (0 < case < 255) with their case index,
 *            same capacity protocol.
 * stats:     optional device gh_stats.
 * Indexed mesh (optional; no counterpart in the paper, which outputs the
 * triangles of Marching Cubes): one vertex per crossing lattice edge,
 * numbered in the order of its lower end point in the pipeline's lattice-
 * vertex list (x, y, z edges in that order), so the numbering does not depend
 * on the triangle order.
 * vert_xyz:  [capacity_verts][3] float32 vertex positions, bit-identical to
 *            the soup's positions of the same edge, or NULL.
 * tri_idx:   [capacity_tris][3] int32 vertex indices of the soup's triangles
 *            (same order and orientation), or NULL; needs tri_keys.
 * n_verts:   one int64 written with the number of vertices; more than
 *            capacity_verts gives GH_ERR_CAPACITY as for triangles.
 * Supported by gh_polygonize and gh_polygonize_batch with GH_METHOD_HOP. */
typedef struct {
    float *tri_xyz;
    uint64_t *tri_keys;
    int64_t capacity_tris;
    int64_t *n_tris;
    uint64_t *cell_ids;
    uint8_t *cell_cases;
    int64_t capacity_cells;
    int64_t *n_cells;
    gh_stats *stats;
    float *vert_xyz;
    int32_t *tri_idx;
    int64_t capacity_verts;
    int64_t *n_verts;
} gh_mesh;

/* Creates an SDB from a host blob (formats above).  Copies the blob to the
 * device of the current CUDA device; for GH_SDB_MLP also derives the BF16
 * tensor-core copy of the weights.  Errors: GH_ERR_ARG for a malformed blob,
 * GH_ERR_CUDA, GH_ERR_DEVICE when the current device is not sm_103. */
int gh_create_sdb(const gh_sdb_desc *desc, gh_sdb **out);

/* Releases an SDB and its device memory.  NULL is accepted.  The caller must
 * make sure no work that uses it is still running.  Its polygonization
 * scratch (hundreds of MB at N = 1024) is kept in a small per-device pool and
 * handed to the next SDB that needs no more (no counterpart in the paper;
 * allocation per object costs milliseconds). */
int gh_destroy_sdb(gh_sdb *sdb);

/* Frees the pooled scratch of destroyed SDBs on every device.  Always GH_OK. */
int gh_release_cache(void);

/* Measures the BF16 evaluation error of a neural SDB (the reduced-precision
 * counterpart of the paper's shrink factor lambda, Sec. 5.2): eps = 2 * max
 * |f_bf16 - f_ref| over n_points seeded uniform points of the grid's volume
 * together with the lattice points a BF16 hopping run of a grid of N/4 (at
 * least 32) cells evaluates next to the surface, f_ref being the split-BF16
 * evaluator (GH_BF16_REFINE_X6; FP32-level accuracy, within ~1e-8 of FP32
 * here, far inside the factor 2).  Stores eps in the SDB (used when
 * gh_options.eps < 0) and, if eps_out is not NULL, writes it to the host
 * float.  Synchronises the stream.  GH_ERR_UNIMPLEMENTED when the SDB's
 * width / depth has no BF16 path. */
int gh_sdb_calibrate(gh_sdb *sdb, const gh_grid *grid, int64_t n_points, uint64_t seed, float *eps_out,
                     void *stream);

/* Polygonizes one SDB on a grid: the paper's apply_grid_hopping(eval_sdb, N)
 * (Algorithm 1) with Marching Cubes filled in at the polygonization step.
 * stream is a cudaStream_t (NULL = legacy default stream).  Asynchronous
 * unless opts->sync; see gh_options.  Errors: GH_ERR_ARG, GH_ERR_CAPACITY
 * (sync only; *n_tris then holds the required count), GH_ERR_NONFINITE,
 * GH_ERR_CUDA. */
int gh_polygonize(const gh_grid *grid, const gh_sdb *sdb, const gh_options *opts, gh_mesh *out, void *stream);

/* Polygonizes B SDBs, each on its own grid (Algorithm 1 for every item).
 * The ray hopping of all analytic items runs in one persistent launch, and
 * that of all neural items of one width in one persistent launch, each fed by
 * device work queues (every CTA walks the items in order and takes columns
 * from the current item's queue); lattice-vertex evaluation of the neural
 * items is batched the same way; lists and Marching Cubes run per item.
 * grids[b], sdbs[b], outs[b] as in gh_polygonize; every item needs its own
 * SDB object (B distinct pointers).  opts->precision applies to the neural
 * items (analytic items always run in FP32); BF16 items use opts->eps when
 * >= 0, else their calibrated eps.
 * graph == NULL: runs the batch on stream (sync / async as opts->sync).
 * graph != NULL: runs the batch once synchronously (sizing the scratch), then
 * captures the same launch sequence into a CUDA graph and writes its
 * cudaGraphExec_t to *graph without running it again; replay it with
 * cudaGraphLaunch on a stream, and release it with gh_batch_graph_free.  The
 * SDBs, grids and output buffers stay bound to the graph. */
int gh_polygonize_batch(int B, const gh_grid *grids, const gh_sdb *const *sdbs, const gh_options *opts,
                        gh_mesh *outs, void *stream, void **graph);

/* Replays a graph made by gh_polygonize_batch on stream (cudaGraphLaunch). */
int gh_batch_graph_launch(void *graph, void *stream);

/* Destroys a graph made by gh_polygonize_batch and the descriptors it uses. */
int gh_batch_graph_free(void *graph);

/* No-allocation variant of gh_polygonize for analytic (CSG) scenes.  The
 * paper has no counterpart: this entry point serves callers that cannot
 * allocate device memory while they polygonize -- a plug-in inside a host
 * application that owns the whole device-memory budget and hands out no
 * more, or a real-time loop that must not call cudaMalloc / cudaFree because
 * those calls can block on, or synchronise with, work already running on the
 * device.  It calls no allocator: its scratch is one file-scope __device__
 * array of GH_NOALLOC_SCRATCH_BYTES bytes, which every GPU that loads this
 * library keeps from load until the process exits.
 *   grid:   as in gh_polygonize, with N <= GH_NOALLOC_MAX_N.
 *   prims:  device array of n_prim gh_csg_prim records (1 <= n_prim <=
 *           GH_MAX_PRIMS); caller-owned, only read (a copy with derived
 *           data is staged in the static array).  They must meet the rules
 *           gh_create_sdb checks; being on the device, they are not checked.
 *   out:    caller-owned device buffers, as in gh_polygonize.
 *   stream: a cudaStream_t (NULL = legacy default stream).
 * The call waits for its stream and reports errors as gh_polygonize with
 * sync = 1 does, except that the scratch never grows: a scene that marks
 * more cells, or needs more lattice vertices, than the array holds returns
 * GH_ERR_CAPACITY with a message giving both numbers; N above the maximum
 * returns GH_ERR_ARG.  The first call on a device looks up the device
 * address of the array (cudaGetSymbolAddress) with that device current and
 * keeps it for later calls; make that first call before any stream capture.
 * The kept address belongs to the device's primary context: after
 * cudaDeviceReset on that device this entry point must not be called again
 * in the process.  Before returning, every call waits for its stream and
 * reads the device counters back to the host (that is how it reports
 * GH_ERR_CAPACITY and GH_ERR_NONFINITE).  Every call uses the same array and
 * leaves its contents behind (each call clears its own counters before use),
 * so calls that overlap on the GPU -- from different streams or threads at
 * the same time -- race; serialise them.  Devices with an ordinal of 64 or
 * more get GH_ERR_DEVICE. */
#define GH_NOALLOC_MAX_N 256
#define GH_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
int gh_polygonize_csg_noalloc(const gh_grid *grid, const gh_csg_prim *prims, int32_t n_prim, int32_t tau_mode,
                              gh_mesh *out, void *stream);

/* Continuation (Sec. 2, the comparison method of Sec. 5.1) for analytic
 * SDBs: the surface is crawled from seed cells instead of hopped.  For each
 * seed point (host float32 seeds[n_seeds][3], 1 <= n_seeds <= 65536) the cell
 * holding it is found, and the lattice vertices of its (j, k) line are scanned
 * in +x order from there: the first sign change gives the seed cell (none
 * when the line has none).  From the seed cells, every cell whose surface
 * crosses a face into a neighbour adds that neighbour (each cell once), and
 * each cell gets Marching Cubes from its own eight corner values -- the
 * evaluator and lattice points of gh_polygonize, so a crawled component's
 * triangles equal gh_polygonize's bit for bit.  Each seed reaches one
 * connected component of the mesh (seeds of one component add nothing).
 * opts: precision GH_FP32 (the only one); sync and the capacity protocol as
 * gh_polygonize; stats->hop_evals counts the evaluations (8 per crawled cell
 * plus the seed searches), marked_cells the crawled cells.  No indexed mesh.
 * Errors: GH_ERR_UNIMPLEMENTED for a neural SDB, others as gh_polygonize. */
int gh_polygonize_cont(const gh_grid *grid, const gh_sdb *sdb, const float *seeds, int32_t n_seeds,
                       const gh_options *opts, gh_mesh *out, void *stream);

/* The order in which the hoppers take the N^2 columns (a column is i*N + j,
 * i along x, j along y): the c-th claim of the queue gets column
 * gh_column_order(N, c).  Square rings around the grid centre, innermost
 * first, so the rays claimed last lie at the domain's edge.  A bijection of
 * [0, N^2); returns -1 for N outside [1, 2048] or c outside [0, N^2).  Host
 * only; no device work. */
int64_t gh_column_order(int32_t N, int64_t c);

/* Implicit-surface adjoint: given mesh vertices v[V][3] (device, float32) and
 * the loss gradient dL/dv[V][3] (device), writes
 *   dL/dtheta = sum_v s_v df/dtheta(v),  s_v = -(dL/dv . grad_x f)/|grad_x f|^2,
 * i.e. dv/dtheta = -grad_x f (df/dtheta) / |grad_x f|^2 for a vertex that
 * stays on the level set f = 0 (a rule the paper does not state; it follows
 * from differentiating f(v(theta); theta) = 0).
 * Neural SDB: dL_dtheta is packed like the MLP blob's parameters; the
 *   activations are recomputed at each vertex.
 * Analytic SDB: dL_dtheta is float32[n_prim][20], laid out like the
 *   gh_csg_prim records: slots 2..4 hold dL/dcentre, 5..7 dL/dparam
 *   (radius; major/minor radius; half sizes), every other slot 0 (rotations
 *   are not differentiated).  Each vertex contributes to the one primitive the
 *   min/max fold selects there.
 * dL_dtheta is device float32 and is overwritten.  Deterministic
 * (fixed-order reductions).  V = 0 gives zeros.  Neural SDBs take the
 * vertices in chunks of GH_ADJOINT_CHUNK (the SDB keeps a work buffer of
 * 2 (n_mid + 1) width floats per chunk vertex); the result is the sum of the
 * chunks' gradients in chunk order, so it equals, bit for bit, the sum of
 * separate calls on those chunks. */
#define GH_ADJOINT_CHUNK 131072
int gh_backward(const gh_sdb *sdb, const float *verts, const float *dL_dv, int64_t V, float *dL_dtheta,
                void *stream);

/* Evaluates f at n points p[n][3] (device float32) into out[n] (device
 * float32) with the given precision -- the evaluator the hopper uses. */
int gh_eval(const gh_sdb *sdb, const float *p, int64_t n, float *out, int32_t precision, void *stream);

/* Profiling aid.  gh_set_profiling(1) makes every later gh_polygonize on the
 * calling thread record CUDA events on its stream around its phases (ray
 * hopping, vertex lists, vertex evaluation, selection of the vertices to
 * refine, FP32 refinement, Marching Cubes).
 * gh_last_profile waits for those events and reports the phase durations of
 * the last call; `launches` (the number of kernels that call launched) is
 * reported whether or not profiling is on. */
#define GH_PHASE_HOP 0
#define GH_PHASE_LISTS 1
#define GH_PHASE_VERTICES 2
#define GH_PHASE_SELECT 3
#define GH_PHASE_REFINE 4
#define GH_PHASE_MC 5
typedef struct {
    int64_t launches;
    int32_t n_phases; /* 6 when timed, 0 when profiling was off */
    int32_t reserved;
    double ms[8];
} gh_profile;
int gh_set_profiling(int enable);
int gh_last_profile(gh_profile *out);

/* The limit, in nanoseconds, of the bounded waits the neural engines make
 * on their own work (BF16 and split-BF16 tensor-core engines: one role waiting
 * for another through an mbarrier; FP32 engine: a weight copy landing).  When
 * a wait runs out the kernel records it, the BF16 engines' roles leave their
 * loops (copies in flight land and issued MMAs complete, with a fixed 2 s
 * limit, before tensor memory is freed) and the FP32 engine records it and
 * keeps waiting for its copy; the call then reports GH_ERR_CUDA ("a bounded
 * device wait timed out") and the SDB stays usable.  Default and maximum 2 s
 * (2e9); 0 makes every such wait run out at once, satisfied or not -- a way
 * to exercise the timeout path.  Process-wide; later launches take it. */
int gh_set_wait_limit_ns(uint64_t ns);

/* Copies the library's Marching Cubes table to host memory: ntri[256] and
 * edges[256][5][3] (-1 padded).  Host-only; needs no GPU. */
int gh_mc_table(int32_t *ntri, int32_t *edges);

/* Number of parameters of a neural SDB blob of this width / depth. */
int64_t gh_mlp_param_count(int32_t width, int32_t n_mid);

/* Thread-local message of the last error (never NULL). */
const char *gh_last_error(void);

/* Library version string. */
const char *gh_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GH_H_ */
