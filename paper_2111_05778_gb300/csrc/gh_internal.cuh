// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/gh.h"

namespace gh {

// Device counters of one polygonization, zeroed at the start of a call.
struct Counters {
    unsigned long long next_col;   // column queue of the hopper
    unsigned long long marks;      // marked cells appended
    unsigned long long hop_evals;  // f evaluations of the rays
    unsigned long long verts;      // unique lattice vertices (set by the line scan)
    unsigned long long refine;     // vertices queued for FP32 re-evaluation
    unsigned long long tris;       // triangles produced
    unsigned long long cells;      // surface cells produced
    unsigned long long flags;      // error bits (FLAG_*)
    unsigned long long next_tile;  // work counter of point-list kernels
    unsigned long long next_tile2; // second work counter (refinement pass)
    unsigned long long row_slots;  // rows the neural hopper ran (live or not): 128 per tile-step
    unsigned long long mesh_verts; // indexed output: crossing lattice edges
    unsigned long long q_head;     // continuation: next queue slot to take
    unsigned long long q_pending;  // continuation: cells queued and not yet finished
    unsigned long long pad[2];
};

enum : unsigned long long {
    FLAG_MARK_OVERFLOW = 1ull,   // marked list exceeded its capacity
    FLAG_VERT_OVERFLOW = 2ull,   // vertex list exceeded its capacity
    FLAG_TRI_OVERFLOW = 4ull,    // caller's triangle buffer too small
    FLAG_CELL_OVERFLOW = 8ull,   // caller's cell buffer too small
    FLAG_NONFINITE = 16ull,      // f was NaN or inf somewhere
    FLAG_TIMEOUT = 32ull,        // a bounded device wait gave up
    FLAG_INDEX_MISS = 64ull,     // indexed output: a triangle edge without a listed end point
};

// Grid parameters as the kernels see them (FP32).
struct GridP {
    int N;
    float lo[3];
    float h;      // (hi - lo) / N
    float inv_h;  // N / (hi - lo)
    float tau;    // polygonization distance
    float eps;    // evaluation error bound subtracted from |f| (0 in FP32)
};

// One CSG primitive, laid out like gh_csg_prim.
struct Prim {
    int type, op;
    float c[3];
    float p[3];
    float rot[9];
    float pad[3];
};
static_assert(sizeof(Prim) == 80, "Prim layout");

// Bounding radius rb of a primitive: the largest distance from its centre to
// a point of the solid, rounded up.  For an exact distance d of a solid
// inside the ball B(c, rb), |p - c| - rb <= d(p) <= |p - c| + rb; the CSG
// evaluator uses the interval to skip primitives that cannot change the
// min / max fold.  The bound is only claimed for the shapes it was derived
// for: positive sizes and an orthonormal rotation (|R R^T - I| <= 1e-6
// entrywise); any other record gets +inf, which turns the skip off.
__host__ __device__ inline float prim_bound_radius(const Prim &q) {
    const double a = q.p[0], b = q.p[1], c = q.p[2];
    double e = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = i == j ? -1.0 : 0.0;
            for (int k = 0; k < 3; ++k) s += (double)q.rot[3 * i + k] * (double)q.rot[3 * j + k];
            e = s > e ? s : (-s > e ? -s : e);
        }
    const bool box = q.type == GH_PRIM_BOX;
    const bool pos = a > 0.0 && (q.type == GH_PRIM_SPHERE || b > 0.0) && (!box || c > 0.0);
    if (!(e <= 1e-6) || !pos) return INFINITY;
    double rb;
    switch (q.type) {
    case GH_PRIM_SPHERE: rb = a; break;
    case GH_PRIM_TORUS: rb = a + b; break;                        // major + minor radius
    case GH_PRIM_BOX: rb = sqrt(a * a + b * b + c * c); break;    // corner
    case GH_PRIM_CAPSULE: rb = a + b; break;                      // half length + radius
    case GH_PRIM_CYLINDER: rb = sqrt(a * a + b * b); break;       // rim (radius, half height)
    case GH_PRIM_HEXPRISM: rb = sqrt(4.0 * a * a / 3.0 + b * b); break;  // corner: circumradius 2a / sqrt(3)
    default: rb = sqrt(a * a + b * b); break;                     // cone: base rim (R, -H)
    }
    return (float)(rb * (1.0 + 1e-6)) + 1e-6f;
}

// Order of the column queue: the c-th claimed column lies on the square ring
// of side s around the grid centre (s = N mod 2, N mod 2 + 2, ...), innermost
// rings first; within a ring, the top row, the bottom row, then the left and
// right columns.  Rays near the middle of the domain, which usually cross
// the surface and hop longest, start first, and the rays claimed last lie
// at the domain's edge, which shortens the tail of the launch when the queue
// runs dry.  A bijection of [0, N^2) for every N >= 1.
__host__ __device__ inline uint32_t column_of_claim(uint32_t c, int N) {
    uint32_t s = (uint32_t)sqrtf((float)c);
    while (s * s > c) --s;
    while ((s + 1) * (s + 1) <= c) ++s;
    ++s;  // smallest side with s * s > c
    if ((s & 1u) != ((uint32_t)N & 1u)) ++s;
    const uint32_t lo = ((uint32_t)N - s) / 2, hi = lo + s - 1;
    if (s == 1) return lo * (uint32_t)N + lo;
    const uint32_t p = c - (s - 2) * (s - 2);
    uint32_t i, j;
    if (p < s) {
        i = lo;
        j = lo + p;
    } else if (p < 2 * s) {
        i = hi;
        j = lo + p - s;
    } else if (p < 3 * s - 2) {
        i = lo + 1 + (p - 2 * s);
        j = lo;
    } else {
        i = lo + 1 + (p - 3 * s + 2);
        j = hi;
    }
    return i * (uint32_t)N + j;
}

// Length of the run of spheres starting at record i that the CSG fold
// combines by min (record 0's op is never used, later records must be
// unions); 0 when record i starts no such run.  The evaluator takes a run's
// minimum in one tight loop (min is exact, so the fold's value is unchanged).
__host__ __device__ inline int prim_sphere_run(const Prim *p, int n, int i) {
    int k = i;
    while (k < n && p[k].type == GH_PRIM_SPHERE && (k == 0 || p[k].op == GH_OP_UNION)) ++k;
    return k - i;
}

// Neural SDB parameters on the device.
struct MlpDev {
    int width, n_mid;
    float r0, alpha, beta, inv_lam;
    float radial;  // 1, or 0 without the |p| term (GH_MLP_NO_RADIAL)
    const float *w0;    // [W][3]
    const float *b0;    // [W]
    const float *wt;    // n_mid x [W(in)][W(out)] transposed FP32 hidden weights
    const float *wtb;   // n_mid x [W(out)][W(in)] FP32 hidden weights, inputs permuted like wt's outputs
    const float *bm;    // n_mid x [W]
    const float *wout;  // [W]
    float bout;
    const uint16_t *wbf;  // n_mid x BF16 hidden weights in the tensor-core tile layout
    const uint16_t *wx6;  // n_mid x 3 BF16 parts (low, middle, high) of the hidden weights, same layout
};

// Scratch of one polygonization (device pointers) and its capacities.
struct Scratch {
    Counters *ctr;
    unsigned long long *marks_raw;  // col | k << 24 | rank << 40
    unsigned long long *marks_csr;  // col | k << 24, grouped by column, k ascending
    uint32_t *colcount;             // [N^2]
    uint32_t *coloff;               // [N^2 + 1]
    uint32_t *linecount;            // [(N+1)^2]
    uint32_t *lineoff;              // [(N+1)^2 + 1]
    uint32_t *blocksum;             // scan partials
    unsigned long long *vkey;       // line | c << 32, grouped by line, c ascending
    float *vval;                    // [cap_verts]
    uint8_t *vflag;                 // [cap_verts] refinement flags
    uint32_t *rlist;                // [cap_verts] vertices to refine
    long long cap_marks, cap_verts;
    float *lat;                     // enumeration: f at all (N+1)^3 lattice points
    long long cap_lat;
    uint32_t *ebase;                // indexed output: first mesh vertex of each list entry [cap_verts + 1]
    uint32_t *ebsum;                // its scan partials
    long long cap_index;            // entries ebase was sized for (0: none)
    uint32_t *vis;                  // continuation: visited bit per cell [N^3 / 32 words]
    long long cap_vis;              // words of vis
};

// One polygonization of a batch: grid, scratch and SDB.  Kernels that serve
// batches walk an array of these; a single call is a batch of one.
struct Item {
    GridP g;
    Scratch s;
    MlpDev m;           // neural SDB (kind 1)
    const Prim *prims;  // analytic SDB (kind 0)
    int nprim;
    int kind;
    gh_mesh out;        // batches: the item's output buffers (single calls pass them as a launch argument)
};

// Packing of mark records.  MARK_EMPTY: the hop value proves that the cell
// holds no zero of f and that all its corner values have one certain sign,
// so the cell is kept in the marked set (it was reached within tau) but its
// corners are not evaluated and Marching Cubes skips it.
constexpr unsigned long long MARK_EMPTY = 1ull << 63;
__host__ __device__ inline unsigned long long pack_mark(uint32_t col, uint32_t k, uint32_t rank, bool empty) {
    return (unsigned long long)col | ((unsigned long long)k << 24) | ((unsigned long long)rank << 40) |
           (empty ? MARK_EMPTY : 0ull);
}
__host__ __device__ inline bool mark_empty(unsigned long long m) { return (m & MARK_EMPTY) != 0ull; }
// d = |f(centre)| - eps at a marked cell centre (x, y, z).  With f
// 1-Lipschitz, |f| >= d - sqrt(3)/2 h at every point of the cell, so when d
// exceeds sqrt(3)/2 h + eps + an FP32 rounding margin the cell has no zero and
// every corner value (BF16 within eps, or FP32) has the sign of f.
__host__ __device__ inline bool cell_is_empty(const GridP &g, float d, float x, float y, float z) {
    return d > 0.8660254f * g.h + g.eps + 1e-5f * (1.f + fabsf(x) + fabsf(y) + fabsf(z));
}
__host__ __device__ inline uint32_t mark_col(unsigned long long m) { return (uint32_t)(m & 0xFFFFFFull); }
__host__ __device__ inline uint32_t mark_k(unsigned long long m) { return (uint32_t)((m >> 24) & 0xFFFFull); }
__host__ __device__ inline uint32_t mark_rank(unsigned long long m) { return (uint32_t)((m >> 40) & 0xFFFFull); }

// The limit of the engines' bounded waits on their own work, in ns (gh_api.cu;
// gh_set_wait_limit_ns; 2 s unless set).
unsigned long long wait_limit_ns();

// ---- launchers implemented in the kernels' translation units ----------------
cudaError_t upload_mc_table(const int32_t *ntri, const int32_t *edges);  // k_pipeline.cu
void launch_init(Scratch &s, cudaStream_t st);
void launch_stage_prims(const Prim *src, Prim *dst, int nprim, cudaStream_t st);  // records + bounding radii
void launch_hop_csg(const Item *items, int n_items, int max_prims, int nsm, int block, cudaStream_t st);
void launch_build_lists(const GridP &g, Scratch &s, cudaStream_t st);
void launch_eval_vertices_csg(const Prim *prims, int nprim, const GridP &g, Scratch &s, int nsm,
                              cudaStream_t st);
void launch_mc(const GridP &g, Scratch &s, const gh_mesh &out, int nsm, cudaStream_t st);
void launch_lattice_csg(const Prim *prims, int nprim, const GridP &g, Scratch &s, cudaStream_t st);
void launch_mc_dense(const GridP &g, Scratch &s, const gh_mesh &out, int nsm, cudaStream_t st);
void launch_enum_stats(const GridP &g, Scratch &s, cudaStream_t st);
void launch_finalize(Scratch &s, const gh_mesh &out, long long columns, cudaStream_t st);
// batches: each per-item step of the pipeline as one launch over all n items
// (every CTA walks the items in order and takes its share of each)
void launch_init_b(const Item *items, int n, cudaStream_t st);
void launch_build_lists_b(const Item *items, int n, int max_N, int nsm, cudaStream_t st);
void launch_eval_vertices_csg_b(const Item *items, int n, int max_prims, int nsm, cudaStream_t st);
void launch_refine_select_b(const Item *items, int n, int nsm, cudaStream_t st);  // neural items only
void launch_mc_b(const Item *items, int n, int nsm, cudaStream_t st);
void launch_finalize_b(const Item *items, int n, cudaStream_t st);
// continuation (Sec. 2) for analytic SDBs: seed search from host-given points
// (seeds: device [n][3]) and the surface crawl with Marching Cubes per cell
void launch_cont_csg(const Prim *prims, int nprim, const GridP &g, Scratch &s, const float *seeds, int n_seeds,
                     const gh_mesh &out, int nsm, cudaStream_t st);
void launch_eval_points_csg(const Prim *prims, int nprim, const float *p, long long n, float *out,
                            cudaStream_t st);

// neural SDB, FP32 on the FFMA pipe (k_mlp_fp32.cu)
void launch_hop_mlp_fp32(const Item *items, int n_items, int width, int nsm, cudaStream_t st);
void launch_eval_vertices_mlp_fp32(const Item *items, int n_items, int width, int nsm, bool refine_list,
                                   cudaStream_t st);
void launch_eval_points_mlp_fp32(const MlpDev &m, const float *p, long long n, float *out, int nsm,
                                 cudaStream_t st);
void launch_lattice_mlp_fp32(const Item *items, int width, int nsm, cudaStream_t st);

// neural SDB, BF16 on tcgen05 tensor cores (k_mlp_bf16.cu)
bool bf16_supported(int width);
int bf16_max_mid(int width);  // hidden layers the BF16 engine supports at this width
void launch_hop_mlp_bf16(const Item *items, int n_items, int width, int nsm, int tiles, cudaStream_t st);
void launch_eval_vertices_mlp_bf16(const Item *items, int n_items, int width, int nsm, int tiles, cudaStream_t st);
void launch_eval_points_mlp_bf16(const MlpDev &m, const float *p, long long n, float *out, int nsm,
                                 cudaStream_t st);
void launch_refine_select(const GridP &g, Scratch &s, cudaStream_t st);  // k_pipeline.cu
// neural SDB with split-BF16 tensor-core products (k_mlp_x6.cu)
int x6_max_mid();
void launch_refine_mlp_x6(const Item *items, int n_items, int width, int nsm, cudaStream_t st);
void launch_eval_points_mlp_x6(const MlpDev &m, const float *p, long long n, float *out, int nsm, cudaStream_t st);
// exclusive scan of n uint32 into out[0..n] (k_pipeline.cu); bsum holds
// ceil(n / 4096) partials; *total gets the sum
void scan_u32_dev(const uint32_t *in, long long n, uint32_t *out, uint32_t *bsum, unsigned long long *total,
                  Counters *ctr, cudaStream_t st);
long long scan_partials(long long n);
// derived weight layouts of a neural SDB from its packed parameters (k_prep.cu)
void launch_prep_mlp(const float *params, int W, int n_mid, float *wt, float *wtb, uint16_t *wbf, uint16_t *wx6,
                     float *bm, cudaStream_t st);
// indexed mesh output after Marching Cubes (k_index.cu)
void launch_index_mesh(const GridP &g, Scratch &s, const gh_mesh &out, int nsm, cudaStream_t st);

// implicit-surface adjoint (k_adjoint.cu)
struct AdjBuffers {
    float *Z, *D, *s, *part, *ones;
    uint32_t *mbits;  // ReLU masks of z_0..z_{L-1}: (VC / 128) tiles x 256 threads x W / 64 words per layer
    int VC, splits, nsm;
};
// the adjoint's forward pass (z_0..z_L of V vertices into Z + l*ldl, masks
// into mbits) and delta chain (delta_L in D + L*ldl down to delta_0),
// k_mlp_fp32.cu
void launch_adj_fwd_fp32(const MlpDev &m, const float *P, long long V, float *Z, long long ldl, uint32_t *mbits,
                         int nsm, cudaStream_t st);
void launch_adj_bwd_fp32(const MlpDev &m, long long V, const uint32_t *mbits, float *D, long long ldl, int nsm,
                         cudaStream_t st);
size_t adjoint_buffer_floats(int W, int n_mid, int VC, int splits);
void adjoint_chunk(const MlpDev &m, const float *P, const float *dL, int V, float *grad, bool accumulate,
                   const AdjBuffers &b, cudaStream_t st);
void adjoint_fill_ones(float *p, long long n, cudaStream_t st);
void csg_adjoint(const Prim *prims, int nprim, const float *V, const float *dL, int nv, int *act, float *contrib,
                 float *out, cudaStream_t st);

// calibration helpers (k_pipeline.cu)
void launch_rand_points(float *p, long long n, const float *lo, float ext, unsigned long long seed, cudaStream_t st);
void launch_vertex_points(const GridP &g, Scratch &s, float *p, cudaStream_t st);
void launch_max_abs_diff(const float *a, const float *b, long long n, unsigned int *out, cudaStream_t st);

}  // namespace gh
