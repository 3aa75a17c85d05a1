// Grid hopping + Marching Cubes pipeline kernels (analytic SDBs and the parts
// shared with the neural SDB).
//
// Pipeline of one polygonization (Sec. 3, Algorithm 1 of the paper, laid out
// for a GPU):
//   1. k_hop_csg      persistent rays, one per lane: evaluate d = |f| at the
//                     cell centre (Eq. 3); d <= tau (Eq. 4) marks the cell and
//                     advances one cell, otherwise the ray jumps floor(d/h)
//                     cells.  Dead lanes are refilled from a column queue
//                     after a warp ballot; marks are appended with one atomic
//                     per warp.
//   2. scans + k_scatter_marks   group the marks by column (k ascending).
//   3. k_lines        for every vertical lattice line, collect the marks of
//                     the (up to) four adjacent columns into the ascending
//                     set of lattice vertices the marked cells need, so each
//                     vertex is evaluated once.
//   4. k_eval_vertices_csg   f at those vertices.
//   5. k_mc           per marked cell: 8 corner values, case index, table
//                     lookup, edge interpolation, warp prefix-sum emit with one
//                     atomic per warp.
#include "gh_internal.cuh"

namespace gh {

__constant__ uint8_t c_tab_n[256];
__constant__ __align__(16) uint8_t c_tab_e[256][16];

cudaError_t upload_mc_table(const int32_t *ntri, const int32_t *edges) {
    uint8_t n[256], e[256][16];
    for (int c = 0; c < 256; ++c) {
        n[c] = (uint8_t)ntri[c];
        for (int t = 0; t < 16; ++t) e[c][t] = 255;
        for (int t = 0; t < 5; ++t)
            for (int v = 0; v < 3; ++v) {
                int x = edges[(c * 5 + t) * 3 + v];
                if (x >= 0) e[c][t * 3 + v] = (uint8_t)x;
            }
    }
    cudaError_t err = cudaMemcpyToSymbol(c_tab_n, n, sizeof(n));
    if (err != cudaSuccess) return err;
    return cudaMemcpyToSymbol(c_tab_e, e, sizeof(e));
}

static constexpr uint32_t NONE = 0xFFFFFFFFu;
static constexpr unsigned FULL = 0xFFFFFFFFu;
static constexpr unsigned long long STOP_FLAGS = FLAG_MARK_OVERFLOW | FLAG_VERT_OVERFLOW;

// ---------------------------------------------------------------------------
// Analytic SDB evaluation: exact distances of the seven primitives of
// Sec. 5.1 (sphere, torus, box, capsule, capped cylinder, hexagonal prism,
// cone), folded with min / max (Sec. 4.2-4.3).  Primitives are read from
// shared memory as five float4 each (all lanes read the same primitive:
// broadcast).
// ---------------------------------------------------------------------------
// Square root on the special-function unit (PTX sqrt.approx.f32, one
// instruction instead of the correctly rounded sequence).  Its error is a
// few units in the last place, far inside the evaluation error budget that
// the results are checked against; every GPU consumer of an analytic SDB
// (hopper, vertex values, point evaluation, enumeration lattice) calls the
// same evaluator, so they agree bit for bit.
__device__ __forceinline__ float fsqrt(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// 2-D signed distance to the regular hexagon of apothem a with edges facing
// 0, 60, ..., 300 degrees: fold into the wedge [-30, 30] degrees, where the
// nearest edge is x = a, |z| <= a / sqrt(3).
__device__ __forceinline__ float hexagon2(float x, float z, float a) {
    x = fabsf(x);
    z = fabsf(z);
    const float mx = -0.5f, mz = 0.8660254037844386f;
    const float dot = fmaf(x, mx, z * mz);
    if (dot > 0.f) {
        x = fmaf(-2.f * dot, mx, x);
        z = fmaf(-2.f * dot, mz, z);
    }
    const float lim = a * 0.5773502691896258f;
    const float v0 = x - a, v1 = z - fminf(fmaxf(z, -lim), lim);
    const float n = fsqrt(fmaf(v0, v0, v1 * v1));
    return v0 < 0.f ? -n : n;
}

// (radius, height) box combination used by the cylinder and the prism
__device__ __forceinline__ float box2(float e0, float e1) {
    const float o0 = fmaxf(e0, 0.f), o1 = fmaxf(e1, 0.f);
    return fsqrt(fmaf(o0, o0, o1 * o1)) + fminf(fmaxf(e0, e1), 0.f);
}

// solid cone, base disc radius R at y = -H, apex at +H; 2-D in (rho, y)
__device__ __forceinline__ float cone2(float rho, float y, float R, float H) {
    const float bs = fminf(fmaxf(rho, 0.f), R);
    const float b0 = rho - bs, b1 = y + H;
    const float db = fsqrt(fmaf(b0, b0, b1 * b1));
    const float e0 = -R, e1 = 2.f * H;
    float t = fmaf(rho - R, e0, (y + H) * e1) / fmaf(e0, e0, e1 * e1);
    t = fminf(fmaxf(t, 0.f), 1.f);
    const float s0 = rho - fmaf(t, e0, R), s1 = y - fmaf(t, e1, -H);
    const float d = fminf(db, fsqrt(fmaf(s0, s0, s1 * s1)));
    const bool inside = y > -H && y < H && rho * 2.f * H < R * (H - y);
    return inside ? -d : d;
}

__device__ __forceinline__ float prim_dist(const float4 *q, float x, float y, float z, int &op) {
    const float4 a = q[0];  // type, op, cx, cy
    const float4 b = q[1];  // cz, p0, p1, p2
    const int type = __float_as_int(a.x);
    op = __float_as_int(a.y);
    const float dx = x - a.z, dy = y - a.w, dz = z - b.x;
    if (type == GH_PRIM_SPHERE) return fsqrt(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) - b.y;
    const float4 r0 = q[2], r1 = q[3], r2 = q[4];  // rot[0..3], rot[4..7], rot[8], pad
    const float lx = fmaf(r0.x, dx, fmaf(r0.y, dy, r0.z * dz));
    const float ly = fmaf(r0.w, dx, fmaf(r1.x, dy, r1.y * dz));
    const float lz = fmaf(r1.z, dx, fmaf(r1.w, dy, r2.x * dz));
    switch (type) {
    case GH_PRIM_TORUS: {
        const float t = fsqrt(fmaf(lx, lx, lz * lz)) - b.y;
        return fsqrt(fmaf(t, t, ly * ly)) - b.z;
    }
    case GH_PRIM_CAPSULE: {
        const float v1 = ly - fminf(fmaxf(ly, -b.y), b.y);
        return fsqrt(fmaf(lx, lx, fmaf(v1, v1, lz * lz))) - b.z;
    }
    case GH_PRIM_CYLINDER: return box2(fsqrt(fmaf(lx, lx, lz * lz)) - b.y, fabsf(ly) - b.z);
    case GH_PRIM_HEXPRISM: return box2(hexagon2(lx, lz, b.y), fabsf(ly) - b.z);
    case GH_PRIM_CONE: return cone2(fsqrt(fmaf(lx, lx, lz * lz)), ly, b.y, b.z);
    default: {
        const float ex = fabsf(lx) - b.y, ey = fabsf(ly) - b.z, ez = fabsf(lz) - b.w;
        const float ox = fmaxf(ex, 0.f), oy = fmaxf(ey, 0.f), oz = fmaxf(ez, 0.f);
        return fsqrt(fmaf(ox, ox, fmaf(oy, oy, oz * oz))) + fminf(fmaxf(ex, fmaxf(ey, ez)), 0.f);
    }
    }
}

// The left fold of Sec. 4.3.  A primitive's distance d lies in
// [|p - c| - rb, |p - c| + rb] (rb: its bounding radius, record slot 17): the
// solid lies in the ball B(c, rb), and d is 1-Lipschitz with |d(c)| <= rb.
// When that interval (widened by a margin far above FP32 rounding) shows that
// min(f, d), max(f, -d) or max(f, d) would return f, the exact distance is
// not evaluated: f is bit-for-bit what the full fold gives.  Spheres are
// always evaluated (their bound costs as much as their distance); a run of
// spheres joined by union (its length in record slot 18) is folded as the
// minimum of the run, in a loop without the per-primitive dispatch.
__device__ __forceinline__ float sphere_run_min(const float4 *P, int i0, int cnt, float x, float y, float z) {
    float m = INFINITY;
#pragma unroll 4
    for (int j = i0; j < i0 + cnt; ++j) {
        const float4 a = P[5 * j], b = P[5 * j + 1];  // type, op, cx, cy | cz, r, -, -
        const float dx = x - a.z, dy = y - a.w, dz = z - b.x;
        m = fminf(m, fsqrt(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) - b.y);
    }
    return m;
}

__device__ __forceinline__ float csg_eval(const float4 *P, int n, float x, float y, float z) {
    int op, i;
    float f;
    const int run0 = __float_as_int(P[4].z);
    if (run0 >= 2) {
        f = sphere_run_min(P, 0, run0, x, y, z);
        i = run0;
    } else {
        f = prim_dist(P, x, y, z, op);
        i = 1;
    }
    for (; i < n; ++i) {
        const float4 *q = P + 5 * i;
        const int run = __float_as_int(q[4].z);
        if (run >= 2) {
            f = fminf(f, sphere_run_min(P, i, run, x, y, z));
            i += run - 1;
            continue;
        }
        const float4 a = q[0], b = q[1];
        const int type = __float_as_int(a.x);
        op = __float_as_int(a.y);
        if (type != GH_PRIM_SPHERE) {
            const float dx = x - a.z, dy = y - a.w, dz = z - b.x;
            const float dc = fsqrt(fmaf(dx, dx, fmaf(dy, dy, dz * dz))), rb = q[4].y;
            const float m = 2e-5f * (dc + rb + fabsf(f) + 1.f);
            const bool skip = op == GH_OP_UNION ? dc - rb >= f + m
                                                : (op == GH_OP_SUBTRACT ? dc - rb >= m - f : dc + rb + m <= f);
            if (skip) continue;
        }
        const float d = prim_dist(q, x, y, z, op);
        f = op == GH_OP_UNION ? fminf(f, d) : (op == GH_OP_SUBTRACT ? fmaxf(f, -d) : fmaxf(f, d));
    }
    return f;
}

// The primitive table is kept as ints in the type/op slots: convert the
// host's gh_csg_prim (int32 type/op) bit-exactly -- they already are ints.
__device__ __forceinline__ void load_prims(float4 *dst, const Prim *src, int nprim) {
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
    for (int i = threadIdx.x; i < nprim * 5; i += blockDim.x) dst[i] = s4[i];
    __syncthreads();
}

// Copy caller-owned primitive records and write the derived slots the
// evaluator reads: pad[0] the bounding radius, pad[1] the union-sphere run
// length; pad[2] is cleared.
__global__ void k_stage_prims(const Prim *__restrict__ src, Prim *__restrict__ dst, int nprim) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nprim) return;
    Prim q = src[i];
    q.pad[0] = prim_bound_radius(q);
    q.pad[1] = __int_as_float(prim_sphere_run(src, nprim, i));
    q.pad[2] = 0.f;
    dst[i] = q;
}

void launch_stage_prims(const Prim *src, Prim *dst, int nprim, cudaStream_t st) {
    k_stage_prims<<<(nprim + 127) / 128, 128, 0, st>>>(src, dst, nprim);
}

// ---------------------------------------------------------------------------
__global__ void k_init(Counters *c) {
    unsigned long long *p = reinterpret_cast<unsigned long long *>(c);
    if (threadIdx.x < sizeof(Counters) / 8) p[threadIdx.x] = 0ull;
}

void launch_init(Scratch &s, cudaStream_t st) { k_init<<<1, 32, 0, st>>>(s.ctr); }

// ---------------------------------------------------------------------------
// 1. Persistent hopper for analytic SDBs over a batch of items.  Lanes take
//    columns of item cur; a warp leaves the item when its lanes are done and
//    the item's queue is empty; the CTA then moves on to the next item
//    together (its primitives are staged in shared memory).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_hop_csg(const Item *__restrict__ items, int n_items) {
    extern __shared__ float4 sprim[];
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    for (int cur = 0; cur < n_items; ++cur) {
        const Item &it = items[cur];
        load_prims(sprim, it.prims, it.nprim);  // ends with __syncthreads
        const int nprim = it.nprim;
        const GridP g = it.g;
        const Scratch &s = it.s;
        const int N = g.N;
        const uint32_t ncols = (uint32_t)N * (uint32_t)N;
        uint32_t col = NONE, rank = 0;
        int k = 0;
        bool done = false;
        float x = 0.f, y = 0.f;
        unsigned long long evals = 0;
        for (;;) {
            const bool need = col == NONE && !done;
            const unsigned needm = __ballot_sync(FULL, need);
            if (needm) {
                const int leader = __ffs(needm) - 1;
                unsigned long long base = 0;
                if (lane == leader) base = atomicAdd(&s.ctr->next_col, (unsigned long long)__popc(needm));
                base = __shfl_sync(FULL, base, leader);
                if (need) {
                    const unsigned long long c = base + __popc(needm & lt);
                    if (c < ncols) {
                        col = column_of_claim((uint32_t)c, N);
                        k = 0;
                        rank = 0;
                        const int i = (int)(col / (uint32_t)N), j = (int)(col - (uint32_t)i * N);
                        x = fmaf((float)i + 0.5f, g.h, g.lo[0]);
                        y = fmaf((float)j + 0.5f, g.h, g.lo[1]);
                    } else {
                        done = true;
                    }
                }
            }
            const bool live = col != NONE;
            if (!__any_sync(FULL, live)) break;
            bool mark = false, empty = false;
            int step = 1;
            if (live) {
                const float z = fmaf((float)k + 0.5f, g.h, g.lo[2]);
                const float f = csg_eval(sprim, nprim, x, y, z);
                ++evals;
                float d = fabsf(f) - g.eps;
                if (!isfinite(f)) {
                    atomicOr(&s.ctr->flags, FLAG_NONFINITE);
                    d = 0.f;
                }
                if (d <= g.tau) {
                    mark = true;
                    empty = cell_is_empty(g, d, x, y, z);
                } else {
                    const float stp = floorf(d * g.inv_h);
                    step = stp < 1.f ? 1 : (stp > (float)N ? N : (int)stp);
                }
            }
            const unsigned mm = __ballot_sync(FULL, mark);
            if (mm) {
                const int leader = __ffs(mm) - 1;
                unsigned long long base = 0;
                if (lane == leader) base = atomicAdd(&s.ctr->marks, (unsigned long long)__popc(mm));
                base = __shfl_sync(FULL, base, leader);
                if (mark) {
                    const unsigned long long idx = base + __popc(mm & lt);
                    if (idx < (unsigned long long)s.cap_marks)
                        s.marks_raw[idx] = pack_mark(col, (uint32_t)k, rank, empty);
                    else
                        atomicOr(&s.ctr->flags, FLAG_MARK_OVERFLOW);
                }
            }
            if (live) {
                if (mark) {
                    ++rank;
                    ++k;
                } else {
                    k += step;
                }
                if (k >= N) {
                    s.colcount[col] = rank;
                    col = NONE;
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) evals += __shfl_xor_sync(FULL, evals, o);
        if (lane == 0 && evals) atomicAdd(&s.ctr->hop_evals, evals);
        __syncthreads();  // the primitives are restaged only after every warp is done
    }
}

void launch_hop_csg(const Item *items, int n_items, int max_prims, int nsm, int block, cudaStream_t st) {
    const size_t smem = (size_t)max_prims * sizeof(Prim);
    if (block != 128 && block != 512) block = 256;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hop_csg, block, smem);
    if (per_sm < 1) per_sm = 1;
    k_hop_csg<<<nsm * per_sm, block, smem, st>>>(items, n_items);
}

// ---------------------------------------------------------------------------
// 2. Exclusive scan of uint32 counts (two passes; out has n + 1 entries and
//    out[n] is the total, also stored in *total when total != NULL).
// ---------------------------------------------------------------------------
static constexpr int SCAN_T = 1024, SCAN_IPT = 4, SCAN_TILE = SCAN_T * SCAN_IPT;

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *wsum, uint32_t &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, t, o);
            if (lane >= o) t += y;
        }
        wsum[lane] = t;
    }
    __syncthreads();
    total = wsum[(blockDim.x >> 5) - 1];
    const uint32_t r = (w ? wsum[w - 1] : 0u) + x - v;
    __syncthreads();
    return r;
}

// One tile of the reduction pass (whole block): bsum[tile] = its sum.
__device__ __forceinline__ void scan_reduce_tile(const uint32_t *__restrict__ in, long long n,
                                                 uint32_t *__restrict__ bsum, long long tile, uint32_t *wsum) {
    const long long base = tile * SCAN_TILE + (long long)threadIdx.x * SCAN_IPT;
    uint32_t v = 0;
    for (int i = 0; i < SCAN_IPT; ++i)
        if (base + i < n) v += in[base + i];
    uint32_t tot;
    block_excl_scan(v, wsum, tot);
    if (threadIdx.x == 0) bsum[tile] = tot;
}

// One tile of the apply pass (whole block); the last tile writes out[n] and *total.
__device__ __forceinline__ void scan_apply_tile(const uint32_t *__restrict__ in, long long n,
                                                const uint32_t *__restrict__ bsum, uint32_t *__restrict__ out,
                                                unsigned long long *total, long long tile, long long ntiles,
                                                uint32_t *wsum, uint32_t *prefix) {
    // prefix of this tile = sum of the partials before it
    uint32_t p = 0;
    for (long long i = threadIdx.x; i < tile; i += blockDim.x) p += bsum[i];
    uint32_t ptot;
    block_excl_scan(p, wsum, ptot);
    if (threadIdx.x == 0) *prefix = ptot;
    __syncthreads();
    const uint32_t pre = *prefix;
    const long long base = tile * SCAN_TILE + (long long)threadIdx.x * SCAN_IPT;
    uint32_t v[SCAN_IPT], sum = 0;
    for (int i = 0; i < SCAN_IPT; ++i) {
        v[i] = base + i < n ? in[base + i] : 0u;
        sum += v[i];
    }
    uint32_t tot;
    uint32_t run = pre + block_excl_scan(sum, wsum, tot);
    for (int i = 0; i < SCAN_IPT; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (tile == ntiles - 1 && threadIdx.x == 0) {
        out[n] = pre + tot;
        if (total) *total = (unsigned long long)(pre + tot);
    }
    __syncthreads();  // *prefix is rewritten by the block's next tile
}

__global__ void __launch_bounds__(SCAN_T) k_scan_reduce(const uint32_t *__restrict__ in, long long n,
                                                         uint32_t *__restrict__ bsum, const Counters *ctr) {
    __shared__ uint32_t wsum[32];
    if (ctr->flags & STOP_FLAGS) return;
    scan_reduce_tile(in, n, bsum, blockIdx.x, wsum);
}

__global__ void __launch_bounds__(SCAN_T) k_scan_apply(const uint32_t *__restrict__ in, long long n,
                                                        const uint32_t *__restrict__ bsum, uint32_t *__restrict__ out,
                                                        unsigned long long *total, Counters *ctr) {
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t prefix;
    if (ctr->flags & STOP_FLAGS) return;
    scan_apply_tile(in, n, bsum, out, total, blockIdx.x, gridDim.x, wsum, &prefix);
}

static void scan_u32(const uint32_t *in, long long n, uint32_t *out, uint32_t *bsum, unsigned long long *total,
                     Counters *ctr, cudaStream_t st) {
    const int nb = (int)((n + SCAN_TILE - 1) / SCAN_TILE);
    k_scan_reduce<<<nb, SCAN_T, 0, st>>>(in, n, bsum, ctr);
    k_scan_apply<<<nb, SCAN_T, 0, st>>>(in, n, bsum, out, total, ctr);
}

void scan_u32_dev(const uint32_t *in, long long n, uint32_t *out, uint32_t *bsum, unsigned long long *total,
                  Counters *ctr, cudaStream_t st) {
    scan_u32(in, n, out, bsum, total, ctr, st);
}

long long scan_partials(long long n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 1; }

// ---------------------------------------------------------------------------
// Marks grouped by column.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void scatter_marks(const Scratch &s, unsigned long long t0, unsigned long long stride) {
    const unsigned long long M = s.ctr->marks;
    for (unsigned long long m = t0; m < M; m += stride) {
        const unsigned long long r = s.marks_raw[m];
        const uint32_t col = mark_col(r);
        s.marks_csr[s.coloff[col] + mark_rank(r)] = r & (0xFFFFFFFFFFull | MARK_EMPTY);
    }
}

__global__ void k_scatter_marks(Scratch s) {
    if (s.ctr->flags & STOP_FLAGS) return;
    scatter_marks(s, blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x, (unsigned long long)gridDim.x * blockDim.x);
}

// ---------------------------------------------------------------------------
// 3. Lattice lines.  Line (a,b), 0 <= a,b <= N, holds the lattice vertices
//    (a,b,c).  A marked cell (i,j,k) needs c = k and c = k+1 on the lines
//    (i,j), (i+1,j), (i,j+1), (i+1,j+1).  Each thread gathers the vertices of
//    one line as a bit set over c = 0..N in shared memory (its own words,
//    interleaved with the other threads' so that equal word indices hit
//    different banks), reading the mark lists of the four columns around the
//    line with independent loads; pass 1 counts the set bits, pass 2 writes
//    the keys in ascending c.
// ---------------------------------------------------------------------------
constexpr int LINES_T = 128;

// the corners c = k, k + 1 of a marked cell (none for a cell marked empty)
__device__ __forceinline__ void set_cells(uint32_t *bits, unsigned long long r) {
    if (mark_empty(r)) return;
    const uint32_t k = mark_k(r);
    bits[(k >> 5) * LINES_T] |= 1u << (k & 31);
    const uint32_t k1 = k + 1;  // k + 1 <= N
    bits[(k1 >> 5) * LINES_T] |= 1u << (k1 & 31);
}

template <bool EMIT>
__device__ __forceinline__ void lines_pass(const GridP &g, const Scratch &s, long long t0, long long stride,
                                           uint32_t *lbits) {
    const int N = g.N, N1 = N + 1, NW = (N1 + 31) >> 5;
    uint32_t *bits = lbits + threadIdx.x;  // word w at bits[w * LINES_T]
    const unsigned long long *__restrict__ mk = s.marks_csr;
    const uint32_t *__restrict__ off = s.coloff;
    const long long nlines = (long long)N1 * N1;
    const unsigned long long cap = (unsigned long long)s.cap_verts;
    for (long long line = t0; line < nlines; line += stride) {
        const int a = (int)(line / N1), b = (int)(line - (long long)a * N1);
        for (int w = 0; w < NW; ++w) bits[w * LINES_T] = 0u;
        for (int di = -1; di <= 0; ++di)
            for (int dj = -1; dj <= 0; ++dj) {
                const int i = a + di, j = b + dj;
                if (i < 0 || j < 0 || i >= N || j >= N) continue;
                const uint32_t col = (uint32_t)i * N + j;
                uint32_t m = off[col];
                const uint32_t e = off[col + 1];
                for (; m + 4 <= e; m += 4) {
                    const unsigned long long r0 = __ldg(mk + m), r1 = __ldg(mk + m + 1), r2 = __ldg(mk + m + 2),
                                             r3 = __ldg(mk + m + 3);
                    set_cells(bits, r0);
                    set_cells(bits, r1);
                    set_cells(bits, r2);
                    set_cells(bits, r3);
                }
                for (; m < e; ++m) set_cells(bits, __ldg(mk + m));
            }
        if (!EMIT) {
            uint32_t cnt = 0;
            for (int w = 0; w < NW; ++w) cnt += (uint32_t)__popc(bits[w * LINES_T]);
            s.linecount[line] = cnt;
        } else {
            unsigned long long o = s.lineoff[line];
            for (int w = 0; w < NW; ++w) {
                uint32_t v = bits[w * LINES_T];
                while (v) {
                    const int bit = __ffs(v) - 1;
                    v &= v - 1;
                    if (o < cap) s.vkey[o] = (unsigned long long)line | ((unsigned long long)(32 * w + bit) << 32);
                    ++o;
                }
            }
        }
    }
}

template <bool EMIT>
__global__ void __launch_bounds__(LINES_T) k_lines(GridP g, Scratch s) {
    extern __shared__ uint32_t lbits[];
    if (s.ctr->flags & STOP_FLAGS) return;
    lines_pass<EMIT>(g, s, blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x, lbits);
}

__global__ void k_check_verts(Scratch s) {
    if (s.ctr->verts > (unsigned long long)s.cap_verts) atomicOr(&s.ctr->flags, FLAG_VERT_OVERFLOW);
}

void launch_build_lists(const GridP &g, Scratch &s, cudaStream_t st) {
    const long long ncols = (long long)g.N * g.N, nlines = (long long)(g.N + 1) * (g.N + 1);
    scan_u32(s.colcount, ncols, s.coloff, s.blocksum, nullptr, s.ctr, st);
    k_scatter_marks<<<1024, 256, 0, st>>>(s);
    const int lb = (int)((nlines + LINES_T - 1) / LINES_T);
    const size_t lsm = (size_t)((g.N + 1 + 31) / 32) * LINES_T * sizeof(uint32_t);  // <= 33 KB at N = 2048
    k_lines<false><<<lb, LINES_T, lsm, st>>>(g, s);
    scan_u32(s.linecount, nlines, s.lineoff, s.blocksum, &s.ctr->verts, s.ctr, st);
    k_check_verts<<<1, 1, 0, st>>>(s);
    k_lines<true><<<lb, LINES_T, lsm, st>>>(g, s);
}

// ---------------------------------------------------------------------------
// 4. f at the unique lattice vertices (analytic SDB).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void vertex_pos(const GridP &g, unsigned long long key, float &x, float &y, float &z) {
    const int N1 = g.N + 1;
    const uint32_t line = (uint32_t)(key & 0xFFFFFFFFull), c = (uint32_t)(key >> 32);
    const uint32_t a = line / (uint32_t)N1, b = line - a * (uint32_t)N1;
    x = fmaf((float)a, g.h, g.lo[0]);
    y = fmaf((float)b, g.h, g.lo[1]);
    z = fmaf((float)c, g.h, g.lo[2]);
}

__device__ __forceinline__ void eval_vertices_csg(const float4 *sprim, int nprim, const GridP &g, const Scratch &s,
                                                  unsigned long long t0, unsigned long long stride) {
    const unsigned long long V = s.ctr->verts;
    for (unsigned long long v = t0; v < V; v += stride) {
        float x, y, z;
        vertex_pos(g, s.vkey[v], x, y, z);
        const float f = csg_eval(sprim, nprim, x, y, z);
        if (!isfinite(f)) atomicOr(&s.ctr->flags, FLAG_NONFINITE);
        s.vval[v] = f;
    }
}

__global__ void __launch_bounds__(256) k_eval_vertices_csg(const Prim *__restrict__ gprims, int nprim, GridP g,
                                                            Scratch s) {
    extern __shared__ float4 sprim[];
    load_prims(sprim, gprims, nprim);
    if (s.ctr->flags & STOP_FLAGS) return;
    eval_vertices_csg(sprim, nprim, g, s, blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x,
                      (unsigned long long)gridDim.x * blockDim.x);
}

void launch_eval_vertices_csg(const Prim *prims, int nprim, const GridP &g, Scratch &s, int nsm,
                              cudaStream_t st) {
    const size_t smem = (size_t)nprim * sizeof(Prim);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_eval_vertices_csg, 256, smem);
    if (per_sm < 1) per_sm = 1;
    k_eval_vertices_csg<<<nsm * per_sm, 256, smem, st>>>(prims, nprim, g, s);
}

__global__ void __launch_bounds__(256) k_eval_points_csg(const Prim *__restrict__ gprims, int nprim,
                                                          const float *__restrict__ p, long long n,
                                                          float *__restrict__ out) {
    extern __shared__ float4 sprim[];
    load_prims(sprim, gprims, nprim);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = csg_eval(sprim, nprim, p[3 * i], p[3 * i + 1], p[3 * i + 2]);
}

void launch_eval_points_csg(const Prim *prims, int nprim, const float *p, long long n, float *out,
                            cudaStream_t st) {
    const size_t smem = (size_t)nprim * sizeof(Prim);
    long long nb = (n + 255) / 256;
    if (nb > 4096) nb = 4096;
    if (nb < 1) nb = 1;
    k_eval_points_csg<<<(int)nb, 256, smem, st>>>(prims, nprim, p, n, out);
}

// ---------------------------------------------------------------------------
// 5. Marching Cubes on the marked cells.
// ---------------------------------------------------------------------------
// List indices of the corners c = k of each lane's marked cell (i, j, k) on
// its four vertical lattice lines (q = ox + 2 oy; corner c = k + 1 is the next
// entry).  Every lane of the warp calls it; valid == false for lanes without
// a cell.  A lane whose cell continues a run of consecutive cells of one
// column in the lanes below takes the indices of the run's first cell plus
// its offset: the corners of a run are consecutive entries of each line's
// list (each list holds every corner of the run once, in ascending c).  The
// first cells of runs search; the four lists advance together in one
// branchless binary search, so the loads of the four lines overlap.
__device__ __forceinline__ void cell_corners(const Scratch &s, int N, bool valid, uint32_t col, int i, int j, int k,
                                             uint32_t (&idx)[4]) {
    const int lane = threadIdx.x & 31;
    const uint32_t pcol = __shfl_up_sync(FULL, col, 1);
    const int pk = __shfl_up_sync(FULL, k, 1);
    const int pvalid = __shfl_up_sync(FULL, (int)valid, 1);
    const bool cont = lane > 0 && valid && pvalid && pcol == col && pk + 1 == k;
    const unsigned heads = __ballot_sync(FULL, valid && !cont);
#pragma unroll
    for (int q = 0; q < 4; ++q) idx[q] = 0;
    if (valid && !cont) {
        const uint32_t N1 = (uint32_t)N + 1u;
        const uint32_t l0 = (uint32_t)i * N1 + (uint32_t)j, l1 = l0 + N1;  // lines (i, j), (i + 1, j)
        const uint32_t a0 = s.lineoff[l0], a1 = s.lineoff[l0 + 1], a2 = s.lineoff[l0 + 2];
        const uint32_t b0 = s.lineoff[l1], b1 = s.lineoff[l1 + 1], b2 = s.lineoff[l1 + 2];
        const uint32_t hi[4] = {a1, b1, a2, b2};
        idx[0] = a0;
        idx[1] = b0;
        idx[2] = a1;
        idx[3] = b1;
        const uint32_t len = max(max(a1 - a0, b1 - b0), max(a2 - a1, b2 - b1));
        // the largest p in [lo, hi) with c(p) <= k: c = k is in every list
        for (uint32_t step = len > 1u ? 1u << (31 - __clz(len - 1u)) : 0u; step; step >>= 1) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t p = idx[q] + step;
                if (p < hi[q] && (uint32_t)(s.vkey[p] >> 32) <= (uint32_t)k) idx[q] = p;
            }
        }
    }
    const unsigned below = heads & (lane == 31 ? FULL : ((2u << lane) - 1u));
    const int hl = below ? 31 - __clz(below) : lane;
    const int hk = __shfl_sync(FULL, k, hl);
#pragma unroll
    for (int q = 0; q < 4; ++q) idx[q] = __shfl_sync(FULL, idx[q], hl) + (uint32_t)(k - hk);
}

// The Marching Cubes table in shared memory: the lanes of a warp look up
// different cases, which the constant bank would serve one address at a time.
struct __align__(16) McTab {
    uint8_t e[256][16];
    uint8_t n[256];
};

// Whole block; ends with __syncthreads.
__device__ __forceinline__ void load_tab(McTab &t) {
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        *reinterpret_cast<uint4 *>(t.e[i]) = *reinterpret_cast<const uint4 *>(c_tab_e[i]);
        t.n[i] = c_tab_n[i];
    }
    __syncthreads();
}

// Triangles a warp stages in shared memory before writing them out: room for
// two per cell on average (32 cells, 9 floats each); a warp whose cells have
// more (up to 5 per cell) writes them directly.  The small buffer leaves room
// for more resident warps, which hide this latency-bound kernel's loads.
constexpr int EMIT_TRIS = 32 * 2;
constexpr int EMIT_STAGE = EMIT_TRIS * 9;

// Case index, triangle table and warp prefix-sum emit of one cell per lane;
// every lane of the warp calls it (valid == false for lanes without a cell).
// The warp's triangles take one contiguous range of the output: each lane
// puts its vertex positions at its offset in the warp's staging buffer, and
// the warp then writes the range with consecutive lanes on consecutive
// floats (coalesced stores).
// Per-block slots for claiming output ranges with one atomic per block
// instead of one per warp (the counters are single addresses every warp of
// the grid would otherwise hit).
struct BlockSlots {
    unsigned long long t[8], c[8], tb[8], cb[8], base_t, base_c;
};

__device__ __forceinline__ void emit_cells(const GridP &g, Counters *ctr, const gh_mesh &out, bool valid, int i, int j,
                                           int k, const float (&fv)[8], float *stage, const McTab &tab,
                                           BlockSlots *bs = nullptr) {
    const int N = g.N, N1 = N + 1;
    const unsigned long long N13 = (unsigned long long)N1 * N1 * N1;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    int cs = 0;
    if (valid) {
#pragma unroll
        for (int b = 0; b < 8; ++b) cs |= (fv[b] < 0.f) << b;
    }
    const bool surf = valid && cs != 0 && cs != 255;
    const int nt = surf ? tab.n[cs] : 0;
    // warp-exclusive prefix sum of the triangle counts, one atomic per warp
    int x = nt;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    const int wtot = __shfl_sync(FULL, x, 31);
    const unsigned sm = __ballot_sync(FULL, surf);
    unsigned long long wbase = 0, cbase = 0;
    if (bs) {
        // the whole block calls: one atomic per counter for all its warps
        const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
        if (lane == 0) {
            bs->t[w] = (unsigned long long)wtot;
            bs->c[w] = (unsigned long long)__popc(sm);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long tt = 0, cc = 0;
            for (int q = 0; q < nw; ++q) {
                bs->tb[q] = tt;
                tt += bs->t[q];
                bs->cb[q] = cc;
                cc += bs->c[q];
            }
            bs->base_t = tt ? atomicAdd(&ctr->tris, tt) : 0ull;
            bs->base_c = cc ? atomicAdd(&ctr->cells, cc) : 0ull;
        }
        __syncthreads();
        wbase = bs->base_t + bs->tb[w];
        cbase = bs->base_c + bs->cb[w];
    } else {
        if (wtot) {
            if (lane == 31) wbase = atomicAdd(&ctr->tris, (unsigned long long)wtot);
            wbase = __shfl_sync(FULL, wbase, 31);
        }
        if (sm) {
            if (lane == 0) cbase = atomicAdd(&ctr->cells, (unsigned long long)__popc(sm));
            cbase = __shfl_sync(FULL, cbase, 0);
        }
    }
    const int loc = x - nt;  // this lane's first triangle within the warp's range
    if (sm && out.cell_ids) {
        if (surf) {
            const unsigned long long ci = cbase + __popc(sm & lt);
            if (ci < (unsigned long long)out.capacity_cells) {
                out.cell_ids[ci] = ((unsigned long long)i * N + j) * N + k;
                out.cell_cases[ci] = (uint8_t)cs;
            }
        }
    }
    if (!wtot) return;
    const unsigned long long cap = (unsigned long long)out.capacity_tris;
    const bool staged = wtot <= EMIT_TRIS;  // warp-uniform
    for (int t = 0; t < nt; ++t) {
        const unsigned long long ti = wbase + (unsigned long long)(loc + t);
        // staged: this triangle's slot in the warp's buffer; otherwise its
        // place in the output (nothing is written beyond the capacity)
        float *pos = staged ? stage + 9 * (loc + t) : (ti < cap ? out.tri_xyz + 9 * ti : nullptr);
        unsigned long long key[3];
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            const int e = tab.e[cs][3 * t + v];
            const int ax = e >> 2, u = e & 1, w = (e >> 1) & 1;
            const int ox = ax == 0 ? 0 : u, oy = ax == 1 ? 0 : (ax == 0 ? u : w), oz = ax == 2 ? 0 : w;
            const int blo = ox + 2 * oy + 4 * oz, bhi = blo + (1 << ax);
            const float fa = fv[blo], fb = fv[bhi];
            const float tt = fa / (fa - fb);
            const int la = i + ox, lb = j + oy, lc = k + oz;
            float px = fmaf((float)la, g.h, g.lo[0]);
            float py = fmaf((float)lb, g.h, g.lo[1]);
            float pz = fmaf((float)lc, g.h, g.lo[2]);
            if (ax == 0) px = fmaf(tt, g.h, px);
            else if (ax == 1) py = fmaf(tt, g.h, py);
            else pz = fmaf(tt, g.h, pz);
            if (pos) {
                pos[3 * v] = px;
                pos[3 * v + 1] = py;
                pos[3 * v + 2] = pz;
            }
            key[v] = (unsigned long long)ax * N13 + (unsigned long long)la +
                     (unsigned long long)N1 * ((unsigned long long)lb + (unsigned long long)N1 * lc);
        }
        if (out.tri_keys && ti < cap) {
            unsigned long long *kd = reinterpret_cast<unsigned long long *>(out.tri_keys) + ti * 3;
            kd[0] = key[0];
            kd[1] = key[1];
            kd[2] = key[2];
        }
    }
    if (!staged) return;
    __syncwarp();
    // the warp's range [wbase, wbase + wtot) of triangles, float by float
    const unsigned long long nf = wbase >= cap ? 0ull : 9ull * ((wbase + wtot > cap ? cap : wbase + wtot) - wbase);
    float *dst = out.tri_xyz + 9 * wbase;
    for (unsigned long long f = lane; f < nf; f += 32) dst[f] = stage[f];
    __syncwarp();  // the buffer is free for the warp's next cells
}

// Marching Cubes on the marked cells; the whole block calls, its cells start
// at b0 and step by stride (multiples of the block size).
__device__ __forceinline__ void mc_cells(const GridP &g, const Scratch &s, const gh_mesh &out, float *stage,
                                         const McTab &tab, BlockSlots *bs, unsigned long long b0,
                                         unsigned long long stride) {
    const unsigned long long M = s.ctr->marks;
    const int N = g.N;
    for (unsigned long long mb = b0; mb < M; mb += stride) {
        const unsigned long long m = mb + threadIdx.x;
        const unsigned long long r = m < M ? s.marks_csr[m] : MARK_EMPTY;
        const bool valid = !mark_empty(r);  // cells marked empty have no triangles
        float fv[8];
        const uint32_t col = mark_col(r);
        const int k = (int)mark_k(r);
        const int i = (int)(col / (uint32_t)N), j = (int)(col - (uint32_t)i * N);
        uint32_t idx[4];
        cell_corners(s, N, valid, col, i, j, k, idx);
        if (valid) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                fv[q] = s.vval[idx[q]];
                fv[q + 4] = s.vval[idx[q] + 1];
            }
        }
        emit_cells(g, s.ctr, out, valid, i, j, k, fv, stage, tab, bs);
    }
}

__global__ void __launch_bounds__(256) k_mc(GridP g, Scratch s, gh_mesh out) {
    __shared__ float stage[8][EMIT_STAGE];
    __shared__ McTab tab;
    __shared__ BlockSlots bs;
    if (s.ctr->flags & STOP_FLAGS) return;
    load_tab(tab);
    mc_cells(g, s, out, stage[threadIdx.x >> 5], tab, &bs, blockIdx.x * (unsigned long long)blockDim.x,
             (unsigned long long)gridDim.x * blockDim.x);
}

// ---------------------------------------------------------------------------
// Enumeration (Sec. 2): f at every lattice point, Marching Cubes on every cell.
// Lattice point (a,b,c) is stored at a + (N+1)(b + (N+1)c).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_lattice_csg(const Prim *__restrict__ gprims, int nprim, GridP g, Scratch s) {
    extern __shared__ float4 sprim[];
    load_prims(sprim, gprims, nprim);
    const long long N1 = g.N + 1, n = N1 * N1 * N1;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        const long long a = v % N1, b = (v / N1) % N1, c = v / (N1 * N1);
        const float f = csg_eval(sprim, nprim, fmaf((float)a, g.h, g.lo[0]), fmaf((float)b, g.h, g.lo[1]),
                                 fmaf((float)c, g.h, g.lo[2]));
        if (!isfinite(f)) atomicOr(&s.ctr->flags, FLAG_NONFINITE);
        s.lat[v] = f;
    }
}

void launch_lattice_csg(const Prim *prims, int nprim, const GridP &g, Scratch &s, cudaStream_t st) {
    const size_t smem = (size_t)nprim * sizeof(Prim);
    k_lattice_csg<<<4096, 256, smem, st>>>(prims, nprim, g, s);
}

__global__ void __launch_bounds__(256) k_mc_dense(GridP g, Scratch s, gh_mesh out) {
    __shared__ float stage[8][EMIT_STAGE];
    __shared__ McTab tab;
    __shared__ BlockSlots bs;
    load_tab(tab);
    const long long N = g.N, N1 = N + 1, n = N * N * N;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long mb = blockIdx.x * (long long)blockDim.x; mb < n; mb += stride) {
        const long long m = mb + threadIdx.x;
        const bool valid = m < n;
        float fv[8];
        int i = 0, j = 0, k = 0;
        if (valid) {
            k = (int)(m % N);
            j = (int)((m / N) % N);
            i = (int)(m / (N * N));
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const long long a = i + (b & 1), bb = j + ((b >> 1) & 1), c = k + ((b >> 2) & 1);
                fv[b] = s.lat[a + N1 * (bb + N1 * c)];
            }
        }
        emit_cells(g, s.ctr, out, valid, i, j, k, fv, stage[threadIdx.x >> 5], tab, &bs);
    }
}

__global__ void k_enum_stats(GridP g, Counters *c) {
    const unsigned long long N = g.N, N1 = N + 1;
    c->hop_evals = N1 * N1 * N1;  // evaluations of the enumeration
    c->marks = N * N * N;         // every cell is polygonized
    c->verts = N1 * N1 * N1;
}

void launch_enum_stats(const GridP &g, Scratch &s, cudaStream_t st) { k_enum_stats<<<1, 1, 0, st>>>(g, s.ctr); }

void launch_mc_dense(const GridP &g, Scratch &s, const gh_mesh &out, int nsm, cudaStream_t st) {
    k_mc_dense<<<nsm * 16, 256, 0, st>>>(g, s, out);
}

// Blocks of 256 threads of `kernel` resident per SM (at least 1): the
// Marching Cubes launches are one wave, each block walking the marks with a
// grid stride.
template <typename K>
static int resident_per_sm(K kernel) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0);
    return per_sm < 1 ? 1 : per_sm;
}

void launch_mc(const GridP &g, Scratch &s, const gh_mesh &out, int nsm, cudaStream_t st) {
    static const int per_sm = resident_per_sm(k_mc);
    k_mc<<<nsm * per_sm, 256, 0, st>>>(g, s, out);
}

// ---------------------------------------------------------------------------
// Continuation (Sec. 2), analytic SDBs: from seed cells the surface is crawled
// cell by cell -- a cell's surface leaves it through exactly the faces whose
// four corners do not all have one sign, so the neighbour across each such
// face is a surface cell and is queued once (visited bit per cell).  Each
// queued cell gets Marching Cubes at once from its own eight corner values
// (the hopper's evaluator at the same lattice points, so the triangles are
// bit-identical to the other methods').  The queue lives in the marks buffer
// (cell id + 1 per slot, 0 = not yet written); persistent warps take tickets
// of 32 future slots (one atomic each), every lane polls its own slot and the
// warp processes the cells as they are pushed; the crawl ends when no cell
// is queued or in work (q_pending == 0).  Waits are bounded (2 s of
// %globaltimer) and idle polling backs off.
// ---------------------------------------------------------------------------
constexpr unsigned long long CONT_WAIT_NS = 2000000000ull;

__device__ __forceinline__ unsigned long long gtimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Marks cell c visited; true when this call did (the caller queues it).
__device__ __forceinline__ bool visit(uint32_t *vis, unsigned long long c) {
    const uint32_t bit = 1u << (uint32_t)(c & 31ull);
    return (atomicOr(vis + (c >> 5), bit) & bit) == 0u;
}

// Queues cell c: false when the queue is full (the overflow flag is set and
// the cell is dropped).  The caller has already counted c as pending, so that
// no worker can finish it before it is counted.
__device__ __forceinline__ bool enqueue(const Scratch &s, unsigned long long c) {
    const unsigned long long slot = atomicAdd(&s.ctr->marks, 1ull);
    if (slot >= (unsigned long long)s.cap_marks) {
        atomicOr(&s.ctr->flags, FLAG_MARK_OVERFLOW);
        return false;
    }
    *reinterpret_cast<volatile unsigned long long *>(s.marks_raw + slot) = c + 1ull;
    return true;
}

// One thread per seed point: the cell holding it, then the first sign change
// along the lattice line (a, j0, k0), a = i0 .. N, in +x order.
__global__ void k_cont_seed(const Prim *__restrict__ gprims, int nprim, GridP g, Scratch s,
                            const float *__restrict__ seeds, int n_seeds) {
    extern __shared__ float4 sprim[];
    load_prims(sprim, gprims, nprim);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_seeds) return;
    const int N = g.N;
    int ijk[3];
    for (int a = 0; a < 3; ++a) {
        const float x = floorf((seeds[3 * t + a] - g.lo[a]) * g.inv_h);
        ijk[a] = x < 0.f ? 0 : (x > (float)(N - 1) ? N - 1 : (int)x);
    }
    const float y = fmaf((float)ijk[1], g.h, g.lo[1]), z = fmaf((float)ijk[2], g.h, g.lo[2]);
    float fp = csg_eval(sprim, nprim, fmaf((float)ijk[0], g.h, g.lo[0]), y, z);
    unsigned long long evals = 1;
    for (int a = ijk[0]; a < N; ++a) {
        const float fn = csg_eval(sprim, nprim, fmaf((float)(a + 1), g.h, g.lo[0]), y, z);
        ++evals;
        if ((fp < 0.f) != (fn < 0.f)) {
            const unsigned long long c = ((unsigned long long)a * N + ijk[1]) * N + ijk[2];
            if (visit(s.vis, c)) {
                atomicAdd(&s.ctr->q_pending, 1ull);
                __threadfence();
                if (!enqueue(s, c)) atomicAdd(&s.ctr->q_pending, ~0ull);  // dropped: uncount it
            }
            break;
        }
        fp = fn;
    }
    atomicAdd(&s.ctr->hop_evals, evals);
}

__global__ void __launch_bounds__(256) k_cont_csg(const Prim *__restrict__ gprims, int nprim, GridP g, Scratch s,
                                                  gh_mesh out) {
    extern __shared__ float4 sprim[];
    __shared__ float stage[8][EMIT_STAGE];
    __shared__ McTab tab;
    load_tab(tab);
    load_prims(sprim, gprims, nprim);
    const int N = g.N;
    const int lane = threadIdx.x & 31;
    const unsigned long long cap = (unsigned long long)s.cap_marks;
    volatile unsigned long long *vq = reinterpret_cast<volatile unsigned long long *>(s.marks_raw);
    volatile Counters *vc = s.ctr;
    unsigned long long evals = 0;
    bool over = false;
    while (!over) {
        // a ticket: the next 32 queue slots, each lane waiting for its own
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&s.ctr->q_head, 32ull);
        base = __shfl_sync(FULL, base, 0);
        if (base >= cap) break;  // beyond the queue: nothing will come
        const unsigned long long slot = base + lane;
        bool done = slot >= cap;
        unsigned long long t0 = gtimer_ns(), seen = 0;  // the wait limit runs while the queue does not grow
        unsigned nap = 32;  // idle polling backs off
        for (;;) {
            const unsigned long long v = done ? 0ull : vq[slot];
            const bool ready = v != 0ull;
            if (__ballot_sync(FULL, ready)) {
                const unsigned long long c = ready ? v - 1ull : 0ull;
                const int k = (int)(c % (unsigned long long)N), j = (int)((c / N) % N);
                const int i = (int)(c / ((unsigned long long)N * N));
                float fv[8];
                if (ready) {
#pragma unroll
                    for (int b = 0; b < 8; ++b) {
                        const float f = csg_eval(sprim, nprim, fmaf((float)(i + (b & 1)), g.h, g.lo[0]),
                                                 fmaf((float)(j + ((b >> 1) & 1)), g.h, g.lo[1]),
                                                 fmaf((float)(k + (b >> 2)), g.h, g.lo[2]));
                        if (!isfinite(f)) atomicOr(&s.ctr->flags, FLAG_NONFINITE);
                        fv[b] = f;
                    }
                    evals += 8;
                }
                emit_cells(g, s.ctr, out, ready, i, j, k, fv, stage[threadIdx.x >> 5], tab);
                // the neighbours across the faces the surface crosses that this
                // cell visits first: counted as pending, then queued
                unsigned long long nb[6];
                int nn = 0;
                if (ready) {
#pragma unroll
                    for (int ax = 0; ax < 3; ++ax)
#pragma unroll
                        for (int side = 0; side < 2; ++side) {
                            int neg = 0;
#pragma unroll
                            for (int b = 0; b < 8; ++b)
                                if (((b >> ax) & 1) == side) neg += fv[b] < 0.f;
                            if (neg == 0 || neg == 4) continue;
                            int n3[3] = {i, j, k};
                            n3[ax] += side ? 1 : -1;
                            if (n3[ax] < 0 || n3[ax] >= N) continue;
                            const unsigned long long nc = ((unsigned long long)n3[0] * N + n3[1]) * N + n3[2];
                            if (visit(s.vis, nc)) nb[nn++] = nc;
                        }
                }
                int cnt = nn;
                for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(FULL, cnt, o);
                if (lane == 0 && cnt) atomicAdd(&s.ctr->q_pending, (unsigned long long)cnt);
                __syncwarp();
                __threadfence();  // counted before any of them can be taken
                long long fin = 0;
                for (int q = 0; q < nn; ++q)
                    if (!enqueue(s, nb[q])) ++fin;  // dropped (queue full): uncounted below
                if (ready) {
                    ++fin;  // this cell is finished
                    done = true;
                }
                __threadfence();  // its queued cells are visible before it leaves the count
                for (int o = 16; o > 0; o >>= 1) fin += __shfl_xor_sync(FULL, fin, o);
                if (lane == 0 && fin) atomicAdd(&s.ctr->q_pending, (unsigned long long)(-fin));
                if (__all_sync(FULL, done)) break;  // the ticket is used up: take the next
                nap = 32;
                continue;
            }
            // nothing arrived: the crawl is over when no cell is queued or in work
            int fin = 0;
            if (lane == 0) {
                fin = vc->q_pending == 0ull || (vc->flags & FLAG_TIMEOUT) ? 1 : 0;
                const unsigned long long tail = vc->marks;
                if (tail != seen) {
                    seen = tail;
                    t0 = gtimer_ns();
                }
                if (!fin && gtimer_ns() - t0 > CONT_WAIT_NS) {
                    atomicOr(&s.ctr->flags, FLAG_TIMEOUT);
                    fin = 1;
                }
            }
            if (__shfl_sync(FULL, fin, 0)) {
                over = true;
                break;
            }
            __nanosleep(nap);
            nap = nap < 1024u ? 2u * nap : 1024u;
        }
    }
    for (int o = 16; o > 0; o >>= 1) evals += __shfl_xor_sync(FULL, evals, o);
    if (lane == 0 && evals) atomicAdd(&s.ctr->hop_evals, evals);
}

void launch_cont_csg(const Prim *prims, int nprim, const GridP &g, Scratch &s, const float *seeds, int n_seeds,
                     const gh_mesh &out, int nsm, cudaStream_t st) {
    const size_t smem = (size_t)nprim * sizeof(Prim);
    const unsigned long long ncell = (unsigned long long)g.N * g.N * g.N;
    cudaMemsetAsync(s.vis, 0, sizeof(uint32_t) * ((ncell + 31) / 32), st);
    // the queue's slots read 0 until written (the scratch holds earlier calls' data)
    cudaMemsetAsync(s.marks_raw, 0, sizeof(unsigned long long) * (size_t)s.cap_marks, st);
    k_cont_seed<<<(n_seeds + 127) / 128, 128, smem, st>>>(prims, nprim, g, s, seeds, n_seeds);
    cudaFuncSetAttribute(k_cont_csg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // one CTA (8 warps) per SM: the crawl's front holds a few thousand cells
    k_cont_csg<<<nsm, 256, smem, st>>>(prims, nprim, g, s, out);
}

// ---------------------------------------------------------------------------
// FP32 refinement of the BF16 path.  Marching Cubes on a cell needs the sign
// of each corner and the value at both ends of each crossing edge.  With
// |f_bf16 - f_fp32| <= eps / 2, a corner whose BF16 value clears +-eps has its
// FP32 sign already, and an edge can cross in FP32 only if its BF16 end
// values differ in sign or one of them lies within eps of 0.  So only the
// endpoints of such edges are re-evaluated in FP32; every other corner keeps
// its BF16 value, of which only the (certain) sign is ever used.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void refine_zero(const Scratch &s, unsigned long long t0, unsigned long long stride) {
    const unsigned long long V = s.ctr->verts;
    for (unsigned long long v = t0; v < V; v += stride) s.vflag[v] = 0;
}

__global__ void k_refine_zero(Scratch s) {
    if (s.ctr->flags & STOP_FLAGS) return;
    refine_zero(s, blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x, (unsigned long long)gridDim.x * blockDim.x);
}

__device__ __forceinline__ void refine_select(const GridP &g, const Scratch &s, unsigned long long t0,
                                              unsigned long long stride) {
    const unsigned long long M = s.ctr->marks;
    // the 12 cube edges as corner pairs (corner b at (b&1, b>>1&1, b>>2&1))
    const uint8_t ea[12] = {0, 2, 4, 6, 0, 1, 4, 5, 0, 1, 2, 3};
    const uint8_t eb[12] = {1, 3, 5, 7, 2, 3, 6, 7, 4, 5, 6, 7};
    // warp-uniform loop (t0 - lane starts the warp's marks; stride is a
    // multiple of 32) so that the warp shares its corner searches
    const int lane = threadIdx.x & 31;
    for (unsigned long long mb = t0 - (unsigned long long)lane; mb < M; mb += stride) {
        const unsigned long long m = mb + (unsigned long long)lane;
        const unsigned long long r = m < M ? s.marks_csr[m] : MARK_EMPTY;
        const bool valid = !mark_empty(r);  // cells marked empty: no corners evaluated, no crossing edge
        const uint32_t col = mark_col(r);
        const int k = (int)mark_k(r);
        const int i = (int)(col / (uint32_t)g.N), j = (int)(col - (uint32_t)i * g.N);
        uint32_t vi[8];
        float fv[8];
        cell_corners(s, g.N, valid, col, i, j, k, *reinterpret_cast<uint32_t(*)[4]>(vi));
        if (!valid) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            vi[q + 4] = vi[q] + 1;
            fv[q] = s.vval[vi[q]];
            fv[q + 4] = s.vval[vi[q] + 1];
        }
        uint32_t need = 0;
#pragma unroll
        for (int e = 0; e < 12; ++e) {
            const float a = fv[ea[e]], b = fv[eb[e]];
            if ((a < 0.f) != (b < 0.f) || fabsf(a) <= g.eps || fabsf(b) <= g.eps)
                need |= (1u << ea[e]) | (1u << eb[e]);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c)
            if (need & (1u << c)) s.vflag[vi[c]] = 1;
    }
}

__global__ void k_refine_select(GridP g, Scratch s) {
    if (s.ctr->flags & STOP_FLAGS) return;
    refine_select(g, s, blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x,
                  (unsigned long long)gridDim.x * blockDim.x);
}

// The vertices flagged for refinement, listed; the whole block calls, its
// vertices start at b0 and step by stride (multiples of the block size); one
// atomic per block claims the block's slots.
__device__ __forceinline__ void refine_compact(const Scratch &s, unsigned long long b0, unsigned long long stride) {
    __shared__ unsigned int wcnt[32], wbase[32];
    __shared__ unsigned long long bbase;
    const unsigned long long V = s.ctr->verts;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (unsigned long long vb = b0; vb < V; vb += stride) {
        const unsigned long long v = vb + threadIdx.x;
        const bool f = v < V && s.vflag[v];
        const unsigned fm = __ballot_sync(FULL, f);
        if (lane == 0) wcnt[w] = (unsigned)__popc(fm);
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned int t = 0;
            for (int q = 0; q < nw; ++q) {
                wbase[q] = t;
                t += wcnt[q];
            }
            bbase = t ? atomicAdd(&s.ctr->refine, (unsigned long long)t) : 0ull;
        }
        __syncthreads();
        if (f) s.rlist[bbase + wbase[w] + __popc(fm & ((1u << lane) - 1u))] = (uint32_t)v;
        __syncthreads();  // the slots are rewritten by the next round
    }
}

__global__ void k_refine_compact(Scratch s) {
    if (s.ctr->flags & STOP_FLAGS) return;
    refine_compact(s, blockIdx.x * (unsigned long long)blockDim.x, (unsigned long long)gridDim.x * blockDim.x);
}

void launch_refine_select(const GridP &g, Scratch &s, cudaStream_t st) {
    k_refine_zero<<<1024, 256, 0, st>>>(s);
    k_refine_select<<<1024, 256, 0, st>>>(g, s);
    k_refine_compact<<<1024, 256, 0, st>>>(s);
}

// ---------------------------------------------------------------------------
// Calibration helpers: seeded uniform points (splitmix64, Steele, Lea and
// Flood 2014), the positions of the lattice vertices in the vertex list, and
// max |a - b|.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__global__ void k_rand_points(float *p, long long n, float lo0, float lo1, float lo2, float ext,
                              unsigned long long seed) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        for (int a = 0; a < 3; ++a) {
            const unsigned long long r = splitmix64(seed * 0x100000001B3ull + (unsigned long long)(3 * i + a));
            const float u = (float)(r >> 40) * (1.0f / 16777216.0f);
            p[3 * i + a] = (a == 0 ? lo0 : (a == 1 ? lo1 : lo2)) + u * ext;
        }
}

void launch_rand_points(float *p, long long n, const float *lo, float ext, unsigned long long seed, cudaStream_t st) {
    k_rand_points<<<1024, 256, 0, st>>>(p, n, lo[0], lo[1], lo[2], ext, seed);
}

__global__ void k_vertex_points(GridP g, Scratch s, float *p) {
    if (s.ctr->flags & STOP_FLAGS) return;
    const unsigned long long V = s.ctr->verts;
    for (unsigned long long v = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; v < V;
         v += (unsigned long long)gridDim.x * blockDim.x) {
        float x, y, z;
        vertex_pos(g, s.vkey[v], x, y, z);
        p[3 * v] = x;
        p[3 * v + 1] = y;
        p[3 * v + 2] = z;
    }
}

void launch_vertex_points(const GridP &g, Scratch &s, float *p, cudaStream_t st) {
    k_vertex_points<<<1024, 256, 0, st>>>(g, s, p);
}

__global__ void k_max_abs_diff(const float *a, const float *b, long long n, unsigned int *out) {
    float mx = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = fabsf(a[i] - b[i]);
        mx = (d > mx || d != d) ? (d != d ? __int_as_float(0x7f800000) : d) : mx;
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(mx));
}

void launch_max_abs_diff(const float *a, const float *b, long long n, unsigned int *out, cudaStream_t st) {
    k_max_abs_diff<<<512, 256, 0, st>>>(a, b, n, out);
}

// ---------------------------------------------------------------------------
// Results: counts, statistics and the status word.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void finalize(const Scratch &s, const gh_mesh &out, long long columns) {
    const Counters c = *s.ctr;
    long long status = GH_OK;
    if (c.flags & FLAG_NONFINITE) status = GH_ERR_NONFINITE;
    if (c.flags & (FLAG_MARK_OVERFLOW | FLAG_VERT_OVERFLOW)) status = GH_ERR_CAPACITY;
    if (c.tris > (unsigned long long)out.capacity_tris) status = GH_ERR_CAPACITY;
    if (out.cell_ids && c.cells > (unsigned long long)out.capacity_cells) status = GH_ERR_CAPACITY;
    if (out.vert_xyz && c.mesh_verts > (unsigned long long)out.capacity_verts) status = GH_ERR_CAPACITY;
    if (c.flags & FLAG_INDEX_MISS) status = GH_ERR_CUDA;
    if (c.flags & FLAG_TIMEOUT) status = GH_ERR_CUDA;  // the other counters are then meaningless
    if (out.n_tris) *out.n_tris = (long long)c.tris;
    if (out.n_verts) *out.n_verts = (long long)c.mesh_verts;
    if (out.n_cells) *out.n_cells = (long long)c.cells;
    if (out.stats) {
        gh_stats *st = out.stats;
        st->status = status;
        st->columns = columns;
        st->hop_evals = (long long)c.hop_evals;
        st->marked_cells = (long long)c.marks;
        st->unique_vertices = (long long)c.verts;
        st->refined_vertices = (long long)c.refine;
        st->surface_cells = (long long)c.cells;
        st->triangles = (long long)c.tris;
        st->row_slots = (long long)c.row_slots;
        st->mesh_vertices = (long long)c.mesh_verts;
    }
}

__global__ void k_finalize(Scratch s, gh_mesh out, long long columns) { finalize(s, out, columns); }

void launch_finalize(Scratch &s, const gh_mesh &out, long long columns, cudaStream_t st) {
    k_finalize<<<1, 1, 0, st>>>(s, out, columns);
}

// ---------------------------------------------------------------------------
// Batches: every per-item step as one launch over all items.  A CTA walks the
// items in order and takes its grid-stride share of each one's work; items
// whose scratch overflowed are skipped (the host grows it and runs again).
// ---------------------------------------------------------------------------
__global__ void k_init_b(const Item *__restrict__ items) {
    unsigned long long *p = reinterpret_cast<unsigned long long *>(items[blockIdx.x].s.ctr);
    if (threadIdx.x < sizeof(Counters) / 8) p[threadIdx.x] = 0ull;
}

void launch_init_b(const Item *items, int n, cudaStream_t st) { k_init_b<<<n, 32, 0, st>>>(items); }

__device__ __forceinline__ bool item_stopped(const Item &it) { return (it.s.ctr->flags & STOP_FLAGS) != 0; }

// which = 0: column counts -> column offsets; 1: line counts -> line offsets (total = vertices)
__global__ void __launch_bounds__(SCAN_T) k_scan_reduce_b(const Item *__restrict__ items, int n, int which) {
    __shared__ uint32_t wsum[32];
    for (int b = 0; b < n; ++b) {
        const Item &it = items[b];
        if (item_stopped(it)) continue;
        const long long N = it.g.N, len = which ? (N + 1) * (N + 1) : N * N;
        const long long nt = (len + SCAN_TILE - 1) / SCAN_TILE;
        for (long long t = blockIdx.x; t < nt; t += gridDim.x)
            scan_reduce_tile(which ? it.s.linecount : it.s.colcount, len, it.s.blocksum, t, wsum);
    }
}

__global__ void __launch_bounds__(SCAN_T) k_scan_apply_b(const Item *__restrict__ items, int n, int which) {
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t prefix;
    for (int b = 0; b < n; ++b) {
        const Item &it = items[b];
        if (item_stopped(it)) continue;
        const long long N = it.g.N, len = which ? (N + 1) * (N + 1) : N * N;
        const long long nt = (len + SCAN_TILE - 1) / SCAN_TILE;
        for (long long t = blockIdx.x; t < nt; t += gridDim.x)
            scan_apply_tile(which ? it.s.linecount : it.s.colcount, len, it.s.blocksum,
                            which ? it.s.lineoff : it.s.coloff, which ? &it.s.ctr->verts : nullptr, t, nt, wsum,
                            &prefix);
    }
}

__global__ void k_scatter_marks_b(const Item *__restrict__ items, int n) {
    for (int b = 0; b < n; ++b) {
        const Item &it = items[b];
        if (item_stopped(it)) continue;
        scatter_marks(it.s, blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x,
                      (unsigned long long)gridDim.x * blockDim.x);
    }
}

template <bool EMIT>
__global__ void __launch_bounds__(LINES_T) k_lines_b(const Item *__restrict__ items, int n) {
    extern __shared__ uint32_t lbits[];
    for (int b = 0; b < n; ++b) {
        const Item &it = items[b];
        if (item_stopped(it)) continue;
        lines_pass<EMIT>(it.g, it.s, blockIdx.x * (long long)blockDim.x + threadIdx.x,
                         (long long)gridDim.x * blockDim.x, lbits);
    }
}

__global__ void k_check_verts_b(const Item *__restrict__ items, int n) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < n && items[b].s.ctr->verts > (unsigned long long)items[b].s.cap_verts)
        atomicOr(&items[b].s.ctr->flags, FLAG_VERT_OVERFLOW);
}

void launch_build_lists_b(const Item *items, int n, int max_N, int nsm, cudaStream_t st) {
    const int grid = nsm * 2;
    k_scan_reduce_b<<<grid, SCAN_T, 0, st>>>(items, n, 0);
    k_scan_apply_b<<<grid, SCAN_T, 0, st>>>(items, n, 0);
    k_scatter_marks_b<<<nsm * 8, 256, 0, st>>>(items, n);
    const size_t lsm = (size_t)((max_N + 1 + 31) / 32) * LINES_T * sizeof(uint32_t);
    k_lines_b<false><<<nsm * 16, LINES_T, lsm, st>>>(items, n);
    k_scan_reduce_b<<<grid, SCAN_T, 0, st>>>(items, n, 1);
    k_scan_apply_b<<<grid, SCAN_T, 0, st>>>(items, n, 1);
    k_check_verts_b<<<(n + 127) / 128, 128, 0, st>>>(items, n);
    k_lines_b<true><<<nsm * 16, LINES_T, lsm, st>>>(items, n);
}

__global__ void __launch_bounds__(256) k_eval_vertices_csg_b(const Item *__restrict__ items, int n) {
    extern __shared__ float4 sprim[];
    for (int b = 0; b < n; ++b) {
        const Item &it = items[b];
        if (it.kind != GH_SDB_CSG) continue;
        load_prims(sprim, it.prims, it.nprim);  // ends with __syncthreads
        if (!item_stopped(it))
            eval_vertices_csg(sprim, it.nprim, it.g, it.s, blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x,
                              (unsigned long long)gridDim.x * blockDim.x);
        __syncthreads();  // the next item's primitives replace these only when every thread is done
    }
}

void launch_eval_vertices_csg_b(const Item *items, int n, int max_prims, int nsm, cudaStream_t st) {
    const size_t smem = (size_t)max_prims * sizeof(Prim);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_eval_vertices_csg_b, 256, smem);
    if (per_sm < 1) per_sm = 1;
    k_eval_vertices_csg_b<<<nsm * per_sm, 256, smem, st>>>(items, n);
}

// phase 0: clear the flags, 1: flag the vertices to refine, 2: list them
__global__ void k_refine_b(const Item *__restrict__ items, int n, int phase) {
    for (int b = 0; b < n; ++b) {
        const Item &it = items[b];
        if (it.kind != GH_SDB_MLP || item_stopped(it)) continue;
        const unsigned long long t0 = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
        const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
        if (phase == 0) refine_zero(it.s, t0, stride);
        else if (phase == 1) refine_select(it.g, it.s, t0, stride);
        else refine_compact(it.s, blockIdx.x * (unsigned long long)blockDim.x, stride);
    }
}

void launch_refine_select_b(const Item *items, int n, int nsm, cudaStream_t st) {
    for (int phase = 0; phase < 3; ++phase) k_refine_b<<<nsm * 8, 256, 0, st>>>(items, n, phase);
}

__global__ void __launch_bounds__(256) k_mc_b(const Item *__restrict__ items, int n) {
    __shared__ float stage[8][EMIT_STAGE];
    __shared__ McTab tab;
    __shared__ BlockSlots bs;
    load_tab(tab);
    for (int b = 0; b < n; ++b) {
        const Item &it = items[b];
        if (item_stopped(it)) continue;
        mc_cells(it.g, it.s, it.out, stage[threadIdx.x >> 5], tab, &bs, blockIdx.x * (unsigned long long)blockDim.x,
                 (unsigned long long)gridDim.x * blockDim.x);
    }
}

void launch_mc_b(const Item *items, int n, int nsm, cudaStream_t st) {
    static const int per_sm = resident_per_sm(k_mc_b);
    k_mc_b<<<nsm * per_sm, 256, 0, st>>>(items, n);
}

__global__ void k_finalize_b(const Item *__restrict__ items, int n) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < n) finalize(items[b].s, items[b].out, (long long)items[b].g.N * items[b].g.N);
}

void launch_finalize_b(const Item *items, int n, cudaStream_t st) {
    k_finalize_b<<<(n + 127) / 128, 128, 0, st>>>(items, n);
}

}  // namespace gh
