// Indexed mesh output: one vertex per crossing lattice edge, triangles as
// vertex indices (the optional vert_xyz / tri_idx outputs of gh_mesh).
//
// A lattice edge leaves its lower end point A along +x, +y or +z and crosses
// the surface when f(A) and f(B) differ in sign (inside <=> f < 0, the tie
// rule of the Marching Cubes pass).  The four cells around a crossing edge
// are sign-change cells, which the hopper marks (Algorithm 1 polygonizes
// every cell the surface passes through), so both end points are in the
// vertex list the pipeline already holds (vkey: grouped by vertical lattice
// line, c ascending) together with their final values (vval).
//
// Numbering: vertex-list order of the lower end point, then axis order x, y,
// z.  It depends only on the set of crossing edges, not on the order in which
// the Marching Cubes kernel emitted its triangles.  Vertex positions use the
// Marching Cubes interpolation t = f(A) / (f(A) - f(B)) from A with the same
// operations, so they are bit-identical to the triangle soup's.
#include "gh_internal.cuh"

namespace gh {

namespace {

constexpr unsigned long long STOPF = FLAG_MARK_OVERFLOW | FLAG_VERT_OVERFLOW;

// index of lattice point c of vertical line `line` in the vertex list, or -1
__device__ __forceinline__ long long find_point(const Scratch &s, uint32_t line, uint32_t c) {
    uint32_t lo = s.lineoff[line], hi = s.lineoff[line + 1];
    if (lo >= hi) return -1;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if ((uint32_t)(s.vkey[mid] >> 32) <= c) lo = mid; else hi = mid;
    }
    return (uint32_t)(s.vkey[lo] >> 32) == c ? (long long)lo : -1;
}

// lattice coordinates of list entry v
__device__ __forceinline__ void point_of(const GridP &g, const Scratch &s, unsigned long long v, uint32_t &a,
                                         uint32_t &b, uint32_t &c, uint32_t &line) {
    const uint32_t N1 = (uint32_t)g.N + 1;
    const unsigned long long key = s.vkey[v];
    line = (uint32_t)(key & 0xFFFFFFFFull);
    c = (uint32_t)(key >> 32);
    a = line / N1;
    b = line - a * N1;
}

// bit ax set when the edge from entry v along +ax crosses; nb[ax] = list
// index of the upper end point (or -1 outside the lattice / not listed)
__device__ __forceinline__ int crossing_mask(const GridP &g, const Scratch &s, unsigned long long v,
                                             long long (&nb)[3]) {
    uint32_t a, b, c, line;
    point_of(g, s, v, a, b, c, line);
    const uint32_t N = (uint32_t)g.N, N1 = N + 1;
    nb[0] = a < N ? find_point(s, line + N1, c) : -1;
    nb[1] = b < N ? find_point(s, line + 1, c) : -1;
    nb[2] = (v + 1 < (unsigned long long)s.lineoff[line + 1] && (uint32_t)(s.vkey[v + 1] >> 32) == c + 1)
                ? (long long)(v + 1)
                : -1;
    const bool neg = s.vval[v] < 0.f;
    int m = 0;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax)
        if (nb[ax] >= 0 && (s.vval[nb[ax]] < 0.f) != neg) m |= 1 << ax;
    return m;
}

// per list entry: crossing mask (into vflag) and its population (into cnt);
// entries past the list get 0 so the scan can run over the capacity
__global__ void __launch_bounds__(256) k_edge_count(GridP g, Scratch s, uint32_t *__restrict__ cnt, long long n) {
    if (s.ctr->flags & STOPF) return;
    const unsigned long long V = s.ctr->verts;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        int m = 0;
        if ((unsigned long long)v < V) {
            long long nb[3];
            m = crossing_mask(g, s, (unsigned long long)v, nb);
            s.vflag[v] = (uint8_t)m;
        }
        cnt[v] = (uint32_t)__popc(m);
    }
}

__global__ void __launch_bounds__(256) k_emit_vertices(GridP g, Scratch s, gh_mesh out) {
    if (s.ctr->flags & STOPF) return;
    const unsigned long long V = s.ctr->verts;
    for (unsigned long long v = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; v < V;
         v += (unsigned long long)gridDim.x * blockDim.x) {
        const int m = s.vflag[v];
        if (!m) continue;
        long long nb[3];
        crossing_mask(g, s, v, nb);
        uint32_t a, b, c, line;
        point_of(g, s, v, a, b, c, line);
        const float fa = s.vval[v];
        unsigned long long id = s.ebase[v];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            if (!(m & (1 << ax))) continue;
            const float fb = s.vval[nb[ax]];
            const float tt = fa / (fa - fb);
            float px = fmaf((float)a, g.h, g.lo[0]);
            float py = fmaf((float)b, g.h, g.lo[1]);
            float pz = fmaf((float)c, g.h, g.lo[2]);
            if (ax == 0) px = fmaf(tt, g.h, px);
            else if (ax == 1) py = fmaf(tt, g.h, py);
            else pz = fmaf(tt, g.h, pz);
            if (id < (unsigned long long)out.capacity_verts) {
                out.vert_xyz[3 * id] = px;
                out.vert_xyz[3 * id + 1] = py;
                out.vert_xyz[3 * id + 2] = pz;
            }
            ++id;
        }
    }
}

// triangle corners: edge key -> lower end point -> its first vertex + rank
__global__ void __launch_bounds__(256) k_tri_index(GridP g, Scratch s, gh_mesh out) {
    if (s.ctr->flags & STOPF) return;
    unsigned long long T = s.ctr->tris;
    if (T > (unsigned long long)out.capacity_tris) T = (unsigned long long)out.capacity_tris;
    const unsigned long long N1 = (unsigned long long)g.N + 1, N13 = N1 * N1 * N1;
    const unsigned long long *keys = reinterpret_cast<const unsigned long long *>(out.tri_keys);
    for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < 3 * T;
         q += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long key = keys[q];
        const int ax = (int)(key / N13);
        const unsigned long long r = key - (unsigned long long)ax * N13;
        const uint32_t la = (uint32_t)(r % N1), lb = (uint32_t)((r / N1) % N1), lc = (uint32_t)(r / (N1 * N1));
        const long long idx = find_point(s, la * (uint32_t)N1 + lb, lc);
        int32_t id = -1;
        if (idx >= 0) {
            const int m = s.vflag[idx];
            id = (int32_t)(s.ebase[idx] + (uint32_t)__popc(m & ((1 << ax) - 1)));
        } else {
            atomicOr(&s.ctr->flags, FLAG_INDEX_MISS);
        }
        out.tri_idx[q] = id;
    }
}

}  // namespace

void launch_index_mesh(const GridP &g, Scratch &s, const gh_mesh &out, int nsm, cudaStream_t st) {
    const long long n = s.cap_verts;
    int nb = (int)((n + 255) / 256);
    if (nb > nsm * 8) nb = nsm * 8;
    if (nb < 1) nb = 1;
    k_edge_count<<<nb, 256, 0, st>>>(g, s, s.rlist, n);
    scan_u32_dev(s.rlist, n, s.ebase, s.ebsum, &s.ctr->mesh_verts, s.ctr, st);
    if (out.vert_xyz) k_emit_vertices<<<nb, 256, 0, st>>>(g, s, out);
    if (out.tri_idx) k_tri_index<<<nsm * 8, 256, 0, st>>>(g, s, out);
}

}  // namespace gh
