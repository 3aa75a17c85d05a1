// Host side of the C ABI declared in include/gh.h: argument checks, device
// set-up, the Marching Cubes table, scratch management and the launch
// sequence of one polygonization.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "gh_internal.cuh"

using namespace gh;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err = "no error";

static int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define GH_CUDA(call)                                                                             \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return fail(GH_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

extern "C" const char *gh_last_error(void) { return g_err.c_str(); }

// The bounded waits of the neural engines (gh.h: gh_set_wait_limit_ns).
static std::atomic<unsigned long long> g_wait_ns{2000000000ull};
unsigned long long gh::wait_limit_ns() { return g_wait_ns.load(std::memory_order_relaxed); }

extern "C" int gh_set_wait_limit_ns(uint64_t ns) {
    if (ns > 2000000000ull) return fail(GH_ERR_ARG, "gh_set_wait_limit_ns: %llu ns is above the 2 s maximum",
                                        (unsigned long long)ns);
    g_wait_ns.store(ns == 0 ? 0ull : ns, std::memory_order_relaxed);
    return GH_OK;
}
extern "C" const char *gh_version(void) { return "gridhop-gb300 0.1 (sm_103a)"; }

extern "C" int64_t gh_column_order(int32_t N, int64_t c) {
    if (N < 1 || N > 2048 || c < 0 || c >= (int64_t)N * N) return -1;
    return (int64_t)column_of_claim((uint32_t)c, N);
}

// ---------------------------------------------------------------------------
// Marching Cubes table.  Rule (the paper prints none): on each cube face,
// walk the four corners counter-clockwise as seen from outside the cube;
// every run of negative corners is cut off by one directed segment that
// starts on the edge where the walk enters the run and ends on the edge where
// it leaves it (so the negative side is on the segment's right seen from
// outside and negative corners are never joined across a face).  The
// segments of a case close into loops; a loop is fanned from its
// smallest-index edge whose fan has no triangle lying inside one face.
// ---------------------------------------------------------------------------
static int32_t t_ntri[256];
static int32_t t_edges[256][5][3];
static bool t_ready = false;
static std::mutex t_mu;

static int corner_of(int x, int y, int z) { return x | (y << 1) | (z << 2); }

// edge between two corners that differ in exactly one coordinate
static int edge_between(int c1, int c2) {
    const int lo = c1 < c2 ? c1 : c2, d = c1 ^ c2;
    const int ax = d == 1 ? 0 : (d == 2 ? 1 : 2);
    int uv[2], n = 0;
    for (int a = 0; a < 3; ++a)
        if (a != ax) uv[n++] = (lo >> a) & 1;
    return 4 * ax + uv[0] + 2 * uv[1];
}

// bit mask of the faces (axis*2 + side) an edge lies on
static int edge_faces(int e) {
    const int ax = e >> 2, u = e & 1, v = (e >> 1) & 1;
    int others[2], n = 0;
    for (int a = 0; a < 3; ++a)
        if (a != ax) others[n++] = a;
    return (1 << (others[0] * 2 + u)) | (1 << (others[1] * 2 + v));
}

static void build_table_host() {
    // counter-clockwise corner order of each face seen from outside
    int ring[6][4];
    for (int ax = 0; ax < 3; ++ax)
        for (int sd = 0; sd < 2; ++sd) {
            const int p = ax == 0 ? 1 : 0, q = ax == 2 ? 1 : 2;
            const int sigma = ax == 1 ? -1 : 1;  // e_p x e_q = sigma * e_ax
            const int pq[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
            const bool ccw = sigma * (2 * sd - 1) > 0;
            for (int t = 0; t < 4; ++t) {
                const int *c = pq[ccw ? t : 3 - t];
                int xyz[3];
                xyz[ax] = sd;
                xyz[p] = c[0];
                xyz[q] = c[1];
                ring[ax * 2 + sd][t] = corner_of(xyz[0], xyz[1], xyz[2]);
            }
        }
    for (int cs = 0; cs < 256; ++cs) {
        int nxt[12];
        for (int e = 0; e < 12; ++e) nxt[e] = -1;
        for (int f = 0; f < 6; ++f) {
            int enter[2], leave[2], ne = 0, nl = 0;
            for (int t = 0; t < 4; ++t) {
                const int a = ring[f][t], b = ring[f][(t + 1) & 3];
                const bool na = (cs >> a) & 1, nb = (cs >> b) & 1;
                if (!na && nb) enter[ne++] = t;
                if (na && !nb) leave[nl++] = t;
            }
            // pair each entry with the first exit after it along the ring
            for (int i = 0; i < ne; ++i) {
                int best = -1, bd = 99;
                for (int j = 0; j < nl; ++j) {
                    const int dist = (leave[j] - enter[i] + 4) & 3;
                    if (dist > 0 && dist < bd) {
                        bd = dist;
                        best = j;
                    }
                }
                const int e1 = edge_between(ring[f][enter[i]], ring[f][(enter[i] + 1) & 3]);
                const int e2 = edge_between(ring[f][leave[best]], ring[f][(leave[best] + 1) & 3]);
                nxt[e1] = e2;
            }
        }
        bool seen[12] = {false};
        int nt = 0;
        for (int e0 = 0; e0 < 12; ++e0) {
            if (nxt[e0] < 0 || seen[e0]) continue;
            int loop[12], n = 0;
            for (int x = e0; !seen[x]; x = nxt[x]) {
                seen[x] = true;
                loop[n++] = x;
            }
            int apex = 0;
            bool found = false;
            for (int cand = 0; cand < 12 && !found; ++cand)
                for (int at = 0; at < n && !found; ++at) {
                    if (loop[at] != cand) continue;
                    bool flat = false;
                    for (int i = 1; i + 1 < n; ++i) {
                        const int m = edge_faces(loop[at]) & edge_faces(loop[(at + i) % n]) &
                                      edge_faces(loop[(at + i + 1) % n]);
                        if (m) flat = true;
                    }
                    if (!flat) {
                        apex = at;
                        found = true;
                    }
                }
            for (int i = 1; i + 1 < n; ++i) {
                t_edges[cs][nt][0] = loop[apex];
                t_edges[cs][nt][1] = loop[(apex + i) % n];
                t_edges[cs][nt][2] = loop[(apex + i + 1) % n];
                ++nt;
            }
        }
        t_ntri[cs] = nt;
        for (int t = nt; t < 5; ++t) t_edges[cs][t][0] = t_edges[cs][t][1] = t_edges[cs][t][2] = -1;
    }
    t_ready = true;
}

static void ensure_table() {
    std::lock_guard<std::mutex> lk(t_mu);
    if (!t_ready) build_table_host();
}

extern "C" int gh_mc_table(int32_t *ntri, int32_t *edges) {
    if (!ntri || !edges) return fail(GH_ERR_ARG, "gh_mc_table: NULL output");
    ensure_table();
    memcpy(ntri, t_ntri, sizeof(t_ntri));
    memcpy(edges, t_edges, sizeof(t_edges));
    return GH_OK;
}

// ---------------------------------------------------------------------------
// per-device set-up
// ---------------------------------------------------------------------------
struct DevInfo {
    bool ready = false;
    int nsm = 0;
};
static DevInfo g_dev[64];
static std::mutex g_dev_mu;

static int ensure_device(int *dev_out, int *nsm_out) {
    int dev = 0;
    GH_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(GH_ERR_DEVICE, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (!g_dev[dev].ready) {
        cudaDeviceProp prop;
        GH_CUDA(cudaGetDeviceProperties(&prop, dev));
        if (prop.major != 10 || prop.minor != 3)
            return fail(GH_ERR_DEVICE, "device %d is sm_%d%d; this library is built for sm_103a only", dev, prop.major,
                        prop.minor);
        ensure_table();
        GH_CUDA(upload_mc_table(&t_ntri[0], &t_edges[0][0][0]));
        g_dev[dev].nsm = prop.multiProcessorCount;
        g_dev[dev].ready = true;
    }
    *dev_out = dev;
    *nsm_out = g_dev[dev].nsm;
    return GH_OK;
}

// ---------------------------------------------------------------------------
// SDB objects
// ---------------------------------------------------------------------------
struct gh_sdb {
    int kind = -1;
    int device = 0;
    float lam = 1.f;
    // CSG
    Prim *d_prims = nullptr;
    int nprim = 0;
    // MLP
    MlpDev mlp{};
    std::vector<void *> dbufs;
    float *d_params = nullptr;  // packed parameters as given (float32)
    int64_t nparam = 0;
    float eps = -1.f;           // calibrated BF16 bound (< 0: none yet)
    // scratch, grown on demand
    Scratch scr{};
    int scr_N = 0;
    float *adj = nullptr;  // adjoint work buffer
    float *seeds = nullptr;  // continuation: seed points on the device
    int cap_seeds = 0;
    size_t adj_floats = 0;
    Item h_item{};           // descriptor of the last single call (host copy)
    Item *d_item = nullptr;  // and on the device
    bool item_valid = false;
    std::mutex mu;
};

// Scratch of destroyed SDBs, kept for the next SDB on the same device: the
// scratch of an N = 1024 polygonization is hundreds of MB, and allocating
// and freeing it per SDB object costs milliseconds.  gh_release_cache frees it.
struct PoolEntry {
    Scratch scr;
    int N, device;
};
static std::mutex g_pool_mu;
static std::vector<PoolEntry> g_pool;
constexpr size_t POOL_MAX = 4;

extern "C" int64_t gh_mlp_param_count(int32_t width, int32_t n_mid) {
    const int64_t W = width;
    return 3 * W + W + (int64_t)n_mid * (W * W + W) + W + 1;
}

template <class T>
static int dev_alloc(gh_sdb *s, T **p, size_t n) {
    void *q = nullptr;
    GH_CUDA(cudaMalloc(&q, n * sizeof(T) + 16));
    s->dbufs.push_back(q);
    *p = (T *)q;
    return GH_OK;
}

static int create_csg(gh_sdb *s, const gh_sdb_desc *d) {
    if (d->blob_bytes < sizeof(gh_csg_header)) return fail(GH_ERR_ARG, "CSG blob shorter than its header");
    gh_csg_header h;
    memcpy(&h, d->blob, sizeof(h));
    if (h.n_prim < 1 || h.n_prim > GH_MAX_PRIMS)
        return fail(GH_ERR_ARG, "CSG n_prim = %d outside [1, %d]", h.n_prim, GH_MAX_PRIMS);
    if (d->blob_bytes != sizeof(h) + (size_t)h.n_prim * sizeof(gh_csg_prim))
        return fail(GH_ERR_ARG, "CSG blob has %zu bytes, expected %zu", d->blob_bytes,
                    sizeof(h) + (size_t)h.n_prim * sizeof(gh_csg_prim));
    std::vector<gh_csg_prim> pr(h.n_prim);
    memcpy(pr.data(), (const char *)d->blob + sizeof(h), pr.size() * sizeof(gh_csg_prim));
    for (int i = 0; i < h.n_prim; ++i) {
        const gh_csg_prim &p = pr[i];
        if (p.type < 0 || p.type > GH_PRIM_CONE) return fail(GH_ERR_ARG, "primitive %d: unknown type %d", i, p.type);
        if (p.op < 0 || p.op > 2) return fail(GH_ERR_ARG, "primitive %d: unknown op %d", i, p.op);
        for (int q = 0; q < 3; ++q)
            if (!isfinite(p.centre[q]) || !isfinite(p.param[q])) return fail(GH_ERR_ARG, "primitive %d: non-finite", i);
        for (int q = 0; q < 9; ++q)
            if (!isfinite(p.rot[q])) return fail(GH_ERR_ARG, "primitive %d: non-finite rotation", i);
        // a rotation keeps the primitive's distance a distance (1-Lipschitz,
        // as hopping requires); a scaled or sheared matrix does not
        double dev = 0.0;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double e = r == c ? -1.0 : 0.0;
                for (int k = 0; k < 3; ++k) e += (double)p.rot[3 * r + k] * (double)p.rot[3 * c + k];
                dev = fmax(dev, fabs(e));
            }
        if (dev > 1e-4)
            return fail(GH_ERR_ARG, "primitive %d: rotation is not orthonormal (|R R^T - I| = %.3g)", i, dev);
        if (p.type == GH_PRIM_CONE && !(p.param[0] > 0.f && p.param[1] > 0.f))
            return fail(GH_ERR_ARG, "primitive %d: cone needs R > 0 and H > 0", i);
        // the shrink factor lambda of Sec. 5.2 applies to analytic SDBs as a
        // scale of the distances: fold it into the primitives' parameters is
        // not possible for min/max of differently scaled terms, so lambda is
        // only accepted as 1 for CSG.
    }
    if (s->lam != 1.f) return fail(GH_ERR_UNIMPLEMENTED, "lipschitz_scale != 1 is supported for neural SDBs only");
    // the device copy keeps derived data in the spare slots: pad[0] the
    // primitive's bounding radius (the evaluator skips primitives that cannot
    // change the fold), pad[1] the length of the union-sphere run it starts
    std::vector<Prim> q(pr.size());
    memcpy(q.data(), pr.data(), pr.size() * sizeof(Prim));
    for (size_t i = 0; i < pr.size(); ++i) {
        const int run = prim_sphere_run(q.data(), (int)q.size(), (int)i);
        pr[i].pad[0] = prim_bound_radius(q[i]);
        memcpy(&pr[i].pad[1], &run, sizeof(run));
        pr[i].pad[2] = 0.f;
    }
    if (dev_alloc(s, &s->d_prims, pr.size())) return GH_ERR_CUDA;
    GH_CUDA(cudaMemcpy(s->d_prims, pr.data(), pr.size() * sizeof(gh_csg_prim), cudaMemcpyHostToDevice));
    s->nprim = h.n_prim;
    return GH_OK;
}

static int create_mlp(gh_sdb *s, const gh_sdb_desc *d) {
    if (d->blob_bytes < sizeof(gh_mlp_header)) return fail(GH_ERR_ARG, "MLP blob shorter than its header");
    gh_mlp_header h;
    memcpy(&h, d->blob, sizeof(h));
    const int W = h.width;
    if (W != 64 && W != 128 && W != 256) return fail(GH_ERR_ARG, "MLP width %d not in {64, 128, 256}", W);
    if (h.n_mid < 1 || h.n_mid > 16) return fail(GH_ERR_ARG, "MLP n_mid %d outside [1, 16]", h.n_mid);
    if (!(h.beta > 0) || !isfinite(h.r0) || !isfinite(h.alpha)) return fail(GH_ERR_ARG, "MLP header values invalid");
    if (h.flags & ~GH_MLP_NO_RADIAL) return fail(GH_ERR_ARG, "MLP header: unknown flags 0x%x", h.flags);
    const int64_t np = gh_mlp_param_count(W, h.n_mid);
    if (d->blob_bytes != sizeof(h) + (size_t)np * sizeof(float))
        return fail(GH_ERR_ARG, "MLP blob has %zu bytes, expected %zu", d->blob_bytes, sizeof(h) + (size_t)np * 4);
    const float *P = (const float *)((const char *)d->blob + sizeof(h));
    for (int64_t i = 0; i < np; ++i)
        if (!isfinite(P[i])) return fail(GH_ERR_NONFINITE, "MLP parameter %lld is not finite", (long long)i);
    const float *wout = P + (size_t)4 * W + (size_t)h.n_mid * ((size_t)W * W + W);
    // the engines' layouts of the hidden weights are derived on the device
    // (k_prep.cu); layer 0, biases of layer 0 and the output layer are read
    // in place from the uploaded block
    const size_t WW = (size_t)W * W;
    float *d_wt, *d_wtb, *d_bm;
    uint16_t *d_wbf, *d_wx6;
    if (dev_alloc(s, &s->d_params, (size_t)np) || dev_alloc(s, &d_wt, (size_t)h.n_mid * WW) ||
        dev_alloc(s, &d_wtb, (size_t)h.n_mid * WW) || dev_alloc(s, &d_bm, (size_t)h.n_mid * W) ||
        dev_alloc(s, &d_wbf, (size_t)h.n_mid * WW) || dev_alloc(s, &d_wx6, (size_t)3 * h.n_mid * WW))
        return GH_ERR_CUDA;
    GH_CUDA(cudaMemcpy(s->d_params, P, sizeof(float) * np, cudaMemcpyHostToDevice));
    launch_prep_mlp(s->d_params, W, h.n_mid, d_wt, d_wtb, d_wbf, d_wx6, d_bm, 0);
    GH_CUDA(cudaGetLastError());
    GH_CUDA(cudaStreamSynchronize(0));  // the layouts are complete before any stream uses them
    const float *d_w0 = s->d_params, *d_b0 = s->d_params + 3 * W;
    const float *d_wout = s->d_params + (size_t)4 * W + (size_t)h.n_mid * (WW + W);
    MlpDev &m = s->mlp;
    m.width = W;
    m.n_mid = h.n_mid;
    m.r0 = h.r0;
    m.radial = (h.flags & GH_MLP_NO_RADIAL) ? 0.f : 1.f;
    m.alpha = h.alpha;
    m.beta = h.beta;
    m.inv_lam = 1.f / s->lam;
    m.w0 = d_w0;
    m.b0 = d_b0;
    m.wt = d_wt;
    m.wtb = d_wtb;
    m.bm = d_bm;
    m.wout = d_wout;
    m.bout = wout[W];
    m.wbf = d_wbf;
    m.wx6 = d_wx6;
    s->nparam = np;
    return GH_OK;
}

extern "C" int gh_release_cache(void) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (PoolEntry &e : g_pool) {
        cudaSetDevice(e.device);
        Scratch &c = e.scr;
        void *ptrs[] = {c.ctr, c.marks_raw, c.marks_csr, c.colcount, c.coloff, c.linecount, c.lineoff,
                        c.blocksum, c.vkey, c.vval, c.vflag, c.rlist, c.lat, c.ebase, c.ebsum, c.vis};
        for (void *p : ptrs)
            if (p) cudaFree(p);
    }
    g_pool.clear();
    cudaSetDevice(cur);
    return GH_OK;
}

extern "C" int gh_create_sdb(const gh_sdb_desc *desc, gh_sdb **out) {
    if (!desc || !out) return fail(GH_ERR_ARG, "gh_create_sdb: NULL argument");
    *out = nullptr;
    if (!desc->blob) return fail(GH_ERR_ARG, "gh_create_sdb: NULL blob");
    int dev, nsm;
    int rc = ensure_device(&dev, &nsm);
    if (rc) return rc;
    gh_sdb *s = new gh_sdb();
    s->device = dev;
    s->lam = desc->lipschitz_scale == 0.f ? 1.f : desc->lipschitz_scale;
    if (!(s->lam >= 1.f) || !isfinite(s->lam)) {
        delete s;
        return fail(GH_ERR_ARG, "lipschitz_scale must be >= 1 (or 0 for 1)");
    }
    s->kind = desc->kind;
    if (desc->kind == GH_SDB_CSG) rc = create_csg(s, desc);
    else if (desc->kind == GH_SDB_MLP) rc = create_mlp(s, desc);
    else rc = fail(GH_ERR_ARG, "unknown SDB kind %d", desc->kind);
    if (rc) {
        gh_destroy_sdb(s);
        return rc;
    }
    *out = s;
    return GH_OK;
}

static void free_scratch(gh_sdb *s) {
    Scratch &c = s->scr;
    void *ptrs[] = {c.ctr, c.marks_raw, c.marks_csr, c.colcount, c.coloff, c.linecount, c.lineoff,
                    c.blocksum, c.vkey, c.vval, c.vflag, c.rlist, c.lat, c.ebase, c.ebsum, c.vis};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    s->scr = Scratch{};
    s->scr_N = 0;
}

extern "C" int gh_destroy_sdb(gh_sdb *s) {
    if (!s) return GH_OK;
    if (s->scr.ctr) {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (g_pool.size() < POOL_MAX) {
            g_pool.push_back(PoolEntry{s->scr, s->scr_N, s->device});
            s->scr = Scratch{};
            s->scr_N = 0;
        }
    }
    free_scratch(s);
    if (s->adj) cudaFree(s->adj);
    if (s->seeds) cudaFree(s->seeds);
    if (s->d_item) cudaFree(s->d_item);
    for (void *p : s->dbufs) cudaFree(p);
    delete s;
    return GH_OK;
}

// Allocates the scratch of an N-grid with at least the given capacities (a
// fresh SDB first takes an adequate one from the pool).
static int ensure_scratch(gh_sdb *s, int N, long long want_marks, long long want_verts) {
    Scratch &c = s->scr;
    if (!c.ctr) {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        for (size_t q = 0; q < g_pool.size(); ++q) {
            const PoolEntry &e = g_pool[q];
            if (e.device == s->device && e.N >= N && e.scr.cap_marks >= want_marks && e.scr.cap_verts >= want_verts) {
                c = e.scr;
                s->scr_N = e.N;
                s->item_valid = false;
                g_pool.erase(g_pool.begin() + (long)q);
                break;
            }
        }
    }
    const bool grid_ok = s->scr_N >= N;
    if (grid_ok && c.cap_marks >= want_marks && c.cap_verts >= want_verts) return GH_OK;
    const int NN = grid_ok ? s->scr_N : N;
    long long cm = c.cap_marks > want_marks ? c.cap_marks : want_marks;
    long long cv = c.cap_verts > want_verts ? c.cap_verts : want_verts;
    float *keep_lat = c.lat;
    const long long keep_cap = c.cap_lat;
    uint32_t *keep_vis = c.vis;
    const long long keep_vcap = c.cap_vis;
    c.lat = nullptr;
    c.vis = nullptr;
    free_scratch(s);
    c.lat = keep_lat;
    c.cap_lat = keep_cap;
    c.vis = keep_vis;
    c.cap_vis = keep_vcap;
    s->item_valid = false;
    const long long ncols = (long long)NN * NN, nlines = (long long)(NN + 1) * (NN + 1);
    GH_CUDA(cudaMalloc((void **)&c.ctr, sizeof(Counters)));
    GH_CUDA(cudaMalloc((void **)&c.marks_raw, sizeof(unsigned long long) * cm));
    GH_CUDA(cudaMalloc((void **)&c.marks_csr, sizeof(unsigned long long) * cm));
    GH_CUDA(cudaMalloc((void **)&c.colcount, sizeof(uint32_t) * ncols));
    GH_CUDA(cudaMalloc((void **)&c.coloff, sizeof(uint32_t) * (ncols + 1)));
    GH_CUDA(cudaMalloc((void **)&c.linecount, sizeof(uint32_t) * nlines));
    GH_CUDA(cudaMalloc((void **)&c.lineoff, sizeof(uint32_t) * (nlines + 1)));
    GH_CUDA(cudaMalloc((void **)&c.blocksum, sizeof(uint32_t) * 4096));
    GH_CUDA(cudaMalloc((void **)&c.vkey, sizeof(unsigned long long) * cv));
    GH_CUDA(cudaMalloc((void **)&c.vval, sizeof(float) * cv));
    GH_CUDA(cudaMalloc((void **)&c.vflag, cv));
    GH_CUDA(cudaMalloc((void **)&c.rlist, sizeof(uint32_t) * cv));
    c.cap_marks = cm;
    c.cap_verts = cv;
    s->scr_N = NN;
    return GH_OK;
}

// The vertex numbering of the indexed mesh output (one entry per list slot).
static int ensure_index(gh_sdb *s) {
    Scratch &c = s->scr;
    if (c.cap_index >= c.cap_verts && c.ebase) return GH_OK;
    if (c.ebase) cudaFree(c.ebase);
    if (c.ebsum) cudaFree(c.ebsum);
    c.ebase = nullptr;
    c.ebsum = nullptr;
    c.cap_index = 0;
    GH_CUDA(cudaMalloc((void **)&c.ebase, sizeof(uint32_t) * (c.cap_verts + 1)));
    GH_CUDA(cudaMalloc((void **)&c.ebsum, sizeof(uint32_t) * scan_partials(c.cap_verts)));
    c.cap_index = c.cap_verts;
    s->item_valid = false;
    return GH_OK;
}

static bool wants_index(const gh_mesh &m) { return m.vert_xyz != nullptr || m.tri_idx != nullptr; }

// The dense lattice array of the enumeration method.
static int ensure_lattice(gh_sdb *s, int N) {
    const long long need = (long long)(N + 1) * (N + 1) * (N + 1);
    if (s->scr.cap_lat >= need) return GH_OK;
    if (s->scr.lat) cudaFree(s->scr.lat);
    s->scr.lat = nullptr;
    s->scr.cap_lat = 0;
    GH_CUDA(cudaMalloc((void **)&s->scr.lat, sizeof(float) * need));
    s->scr.cap_lat = need;
    s->item_valid = false;
    return GH_OK;
}

static Item make_item(const gh_sdb *s, const GridP &g) {
    Item it{};  // zero-initialised, padding included, so descriptors compare bytewise
    it.g = g;
    it.s = s->scr;
    it.m = s->mlp;
    it.prims = s->d_prims;
    it.nprim = s->nprim;
    it.kind = s->kind;
    return it;
}

// Uploads the SDB's single-call descriptor when it changed.
static int sync_item(gh_sdb *s, const GridP &g, cudaStream_t st) {
    const Item it = make_item(s, g);
    if (!s->d_item) GH_CUDA(cudaMalloc((void **)&s->d_item, sizeof(Item)));
    if (!s->item_valid || memcmp(&it, &s->h_item, sizeof(Item)) != 0) {
        s->h_item = it;
        GH_CUDA(cudaMemcpyAsync(s->d_item, &s->h_item, sizeof(Item), cudaMemcpyHostToDevice, st));
        GH_CUDA(cudaStreamSynchronize(st));
        s->item_valid = true;
    }
    return GH_OK;
}

// ---------------------------------------------------------------------------
// polygonization
// ---------------------------------------------------------------------------
static int check_grid(const gh_grid *g, GridP *gp, int tau_mode) {
    if (!g) return fail(GH_ERR_ARG, "NULL grid");
    if (g->N < 2 || g->N > 2048) return fail(GH_ERR_ARG, "grid N = %d outside [2, 2048]", g->N);
    float ext[3];
    for (int a = 0; a < 3; ++a) {
        if (!isfinite(g->lo[a]) || !isfinite(g->hi[a])) return fail(GH_ERR_ARG, "grid bounds not finite");
        ext[a] = g->hi[a] - g->lo[a];
        if (!(ext[a] > 0)) return fail(GH_ERR_ARG, "grid: hi must exceed lo on every axis");
    }
    for (int a = 1; a < 3; ++a)
        if (fabsf(ext[a] - ext[0]) > 1e-6f * ext[0])
            return fail(GH_ERR_ARG, "grid must be a cube (equal extents on all axes)");
    if (tau_mode != GH_TAU_DIAGONAL && tau_mode != GH_TAU_HALF_DIAGONAL)
        return fail(GH_ERR_ARG, "unknown tau_mode %d", tau_mode);
    gp->N = g->N;
    for (int a = 0; a < 3; ++a) gp->lo[a] = g->lo[a];
    gp->h = ext[0] / (float)g->N;
    gp->inv_h = (float)g->N / ext[0];
    gp->tau = (float)(sqrt(3.0) * (double)gp->h * (tau_mode == GH_TAU_DIAGONAL ? 1.0 : 0.5));
    gp->eps = 0.f;
    return GH_OK;
}

static int check_mesh(const gh_mesh *m) {
    if (!m) return fail(GH_ERR_ARG, "NULL mesh");
    if (m->capacity_tris < 0 || (m->capacity_tris > 0 && !m->tri_xyz))
        return fail(GH_ERR_ARG, "mesh: tri_xyz is NULL or capacity negative");
    if (m->cell_ids && (!m->cell_cases || m->capacity_cells < 0))
        return fail(GH_ERR_ARG, "mesh: cell_ids given without cell_cases / capacity");
    if (m->tri_idx && !m->tri_keys) return fail(GH_ERR_ARG, "mesh: tri_idx needs tri_keys");
    if (m->vert_xyz && m->capacity_verts < 0) return fail(GH_ERR_ARG, "mesh: capacity_verts negative");
    return GH_OK;
}

// ---------------------------------------------------------------------------
// profiling: CUDA events on the launching stream around each phase
// ---------------------------------------------------------------------------
struct ProfState {
    bool enabled = false;
    bool recorded = false;
    cudaEvent_t ev[7] = {};
    long long launches = 0;
};
static thread_local ProfState g_prof;

extern "C" int gh_set_profiling(int enable) {
    g_prof.enabled = enable != 0;
    if (g_prof.enabled && !g_prof.ev[0])
        for (auto &e : g_prof.ev) GH_CUDA(cudaEventCreate(&e));
    return GH_OK;
}

extern "C" int gh_last_profile(gh_profile *out) {
    if (!out) return fail(GH_ERR_ARG, "gh_last_profile: NULL");
    memset(out, 0, sizeof(*out));
    out->launches = g_prof.launches;
    if (!g_prof.recorded) return GH_OK;
    GH_CUDA(cudaEventSynchronize(g_prof.ev[6]));
    for (int p = 0; p < 6; ++p) {
        float ms = 0.f;
        GH_CUDA(cudaEventElapsedTime(&ms, g_prof.ev[p], g_prof.ev[p + 1]));
        out->ms[p] = ms;
    }
    out->n_phases = 6;
    return GH_OK;
}

static inline void mark_phase(int i, cudaStream_t st) {
    if (g_prof.enabled) cudaEventRecord(g_prof.ev[i], st);
}

// Kernel launches per phase (fixed by the launch sequence below).
static constexpr int LAUNCHES_HOP = 2, LAUNCHES_LISTS = 8, LAUNCHES_VERTS = 1, LAUNCHES_REFINE = 4,
                     LAUNCHES_MC = 2;

static int enqueue_once(gh_sdb *s, const GridP &g, const gh_options &o, const gh_mesh &out, int nsm,
                        cudaStream_t st) {
    Scratch &c = s->scr;
    int rc = sync_item(s, g, st);
    if (rc) return rc;
    long long launches = LAUNCHES_HOP + LAUNCHES_LISTS + LAUNCHES_VERTS + LAUNCHES_MC;
    const int tiles = o.mlp_tiles == 1 ? 1 : 2;
    mark_phase(0, st);
    launch_init(c, st);
    if (o.method == GH_METHOD_ENUM) {
        // Sec. 2 enumeration: every lattice point, every cell
        if (s->kind == GH_SDB_CSG) launch_lattice_csg(s->d_prims, s->nprim, g, c, st);
        else launch_lattice_mlp_fp32(s->d_item, s->mlp.width, nsm, st);
        launch_enum_stats(g, c, st);
        for (int p = 1; p <= 5; ++p) mark_phase(p, st);
        launch_mc_dense(g, c, out, nsm, st);
        launch_finalize(c, out, (long long)g.N * g.N, st);
        mark_phase(6, st);
        g_prof.recorded = g_prof.enabled;
        g_prof.launches = 5;
        GH_CUDA(cudaGetLastError());
        return GH_OK;
    }
    if (s->kind == GH_SDB_CSG) {
        launch_hop_csg(s->d_item, 1, s->nprim, nsm, o.ray_block, st);
        mark_phase(1, st);
        launch_build_lists(g, c, st);
        mark_phase(2, st);
        launch_eval_vertices_csg(s->d_prims, s->nprim, g, c, nsm, st);
        mark_phase(3, st);
        mark_phase(4, st);
        mark_phase(5, st);
    } else if (o.precision == GH_FP32) {
        launch_hop_mlp_fp32(s->d_item, 1, s->mlp.width, nsm, st);
        mark_phase(1, st);
        launch_build_lists(g, c, st);
        mark_phase(2, st);
        launch_eval_vertices_mlp_fp32(s->d_item, 1, s->mlp.width, nsm, false, st);
        mark_phase(3, st);
        mark_phase(4, st);
        mark_phase(5, st);
    } else {
        launch_hop_mlp_bf16(s->d_item, 1, s->mlp.width, nsm, tiles, st);
        mark_phase(1, st);
        launch_build_lists(g, c, st);
        mark_phase(2, st);
        launch_eval_vertices_mlp_bf16(s->d_item, 1, s->mlp.width, nsm, tiles, st);
        mark_phase(3, st);
        launch_refine_select(g, c, st);
        mark_phase(4, st);
        if (o.precision == GH_BF16_REFINE_X6) launch_refine_mlp_x6(s->d_item, 1, s->mlp.width, nsm, st);
        else launch_eval_vertices_mlp_fp32(s->d_item, 1, s->mlp.width, nsm, true, st);
        mark_phase(5, st);
        launches += LAUNCHES_REFINE;
    }
    launch_mc(g, c, out, nsm, st);
    if (wants_index(out)) launch_index_mesh(g, c, out, nsm, st);
    launch_finalize(c, out, (long long)g.N * g.N, st);
    mark_phase(6, st);
    g_prof.recorded = g_prof.enabled;
    g_prof.launches = launches;
    GH_CUDA(cudaGetLastError());
    return GH_OK;
}

extern "C" int gh_polygonize(const gh_grid *grid, const gh_sdb *csdb, const gh_options *opts, gh_mesh *out,
                             void *stream) {
    gh_sdb *s = const_cast<gh_sdb *>(csdb);
    if (!s) return fail(GH_ERR_ARG, "NULL sdb");
    gh_options o{GH_FP32, GH_TAU_DIAGONAL, -1.f, 1, 0, 0, GH_METHOD_HOP};
    if (opts) o = *opts;
    GridP g;
    int rc = check_grid(grid, &g, o.tau_mode);
    if (rc) return rc;
    if ((rc = check_mesh(out))) return rc;
    if (o.method != GH_METHOD_HOP && o.method != GH_METHOD_ENUM) return fail(GH_ERR_ARG, "unknown method %d", o.method);
    if (o.method == GH_METHOD_ENUM && o.precision != GH_FP32)
        return fail(GH_ERR_UNIMPLEMENTED, "the enumeration method runs in FP32 only");
    if (o.method == GH_METHOD_ENUM && wants_index(*out))
        return fail(GH_ERR_UNIMPLEMENTED, "the indexed mesh output needs GH_METHOD_HOP");
    if (o.precision != GH_FP32 && o.precision != GH_BF16_REFINE && o.precision != GH_BF16_REFINE_X6)
        return fail(GH_ERR_ARG, "unknown precision %d", o.precision);
    if (o.precision != GH_FP32) {
        if (s->kind != GH_SDB_MLP) return fail(GH_ERR_ARG, "the BF16 precisions apply to neural SDBs only");
        if (!bf16_supported(s->mlp.width))
            return fail(GH_ERR_UNIMPLEMENTED, "BF16 tensor-core path not available for width %d", s->mlp.width);
        if (s->mlp.n_mid > bf16_max_mid(s->mlp.width))
            return fail(GH_ERR_UNIMPLEMENTED, "BF16 tensor-core path supports at most %d hidden layers at this width",
                        bf16_max_mid(s->mlp.width));
        const float eps = o.eps >= 0.f ? o.eps : s->eps;
        if (!(eps >= 0.f)) return fail(GH_ERR_ARG, "BF16 path needs eps: pass opts.eps or call gh_sdb_calibrate");
        g.eps = eps;
    }
    int dev, nsm;
    if ((rc = ensure_device(&dev, &nsm))) return rc;
    if (dev != s->device) return fail(GH_ERR_ARG, "SDB lives on device %d, current device is %d", s->device, dev);
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(s->mu);
    const long long N2 = (long long)g.N * g.N;
    long long want_m = 8 * N2 > (1 << 16) ? 8 * N2 : (1 << 16);
    long long want_v = 2 * want_m;
    for (int attempt = 0; attempt < 4; ++attempt) {
        if ((rc = ensure_scratch(s, g.N, want_m, want_v))) return rc;
        if (o.method == GH_METHOD_ENUM && (rc = ensure_lattice(s, g.N))) return rc;
        if (wants_index(*out) && (rc = ensure_index(s))) return rc;
        if ((rc = enqueue_once(s, g, o, *out, nsm, st))) return rc;
        if (!o.sync) return GH_OK;
        Counters c;
        GH_CUDA(cudaMemcpyAsync(&c, s->scr.ctr, sizeof(c), cudaMemcpyDeviceToHost, st));
        GH_CUDA(cudaStreamSynchronize(st));
        // a wait that ran out leaves the other counters meaningless
        if (c.flags & FLAG_TIMEOUT) return fail(GH_ERR_CUDA, "a bounded device wait timed out");
        if (c.flags & (FLAG_MARK_OVERFLOW | FLAG_VERT_OVERFLOW)) {
            if (c.flags & FLAG_MARK_OVERFLOW) want_m = (long long)(c.marks + c.marks / 4 + 1024);
            want_v = (c.flags & FLAG_VERT_OVERFLOW) ? (long long)(c.verts + c.verts / 4 + 1024) : 2 * want_m;
            if (want_v < 2 * want_m) want_v = 2 * want_m;
            continue;
        }
        if (c.flags & FLAG_NONFINITE) return fail(GH_ERR_NONFINITE, "the SDB evaluated to NaN or inf");
        if (c.tris > (unsigned long long)out->capacity_tris)
            return fail(GH_ERR_CAPACITY, "triangle buffer holds %lld, %llu needed", (long long)out->capacity_tris,
                        c.tris);
        if (out->cell_ids && c.cells > (unsigned long long)out->capacity_cells)
            return fail(GH_ERR_CAPACITY, "cell buffer holds %lld, %llu needed", (long long)out->capacity_cells,
                        c.cells);
        if (c.flags & FLAG_INDEX_MISS) return fail(GH_ERR_CUDA, "indexed output: a triangle edge was not listed");
        if (out->vert_xyz && c.mesh_verts > (unsigned long long)out->capacity_verts)
            return fail(GH_ERR_CAPACITY, "vertex buffer holds %lld, %llu needed", (long long)out->capacity_verts,
                        c.mesh_verts);
        return GH_OK;
    }
    return fail(GH_ERR_CAPACITY, "internal scratch kept overflowing");
}

// The visited bits of the continuation method (N^3 bits).
static int ensure_vis(gh_sdb *s, int N) {
    const long long need = ((long long)N * N * N + 31) / 32;
    if (s->scr.cap_vis >= need) return GH_OK;
    if (s->scr.vis) cudaFree(s->scr.vis);
    s->scr.vis = nullptr;
    s->scr.cap_vis = 0;
    GH_CUDA(cudaMalloc((void **)&s->scr.vis, sizeof(uint32_t) * need));
    s->scr.cap_vis = need;
    s->item_valid = false;
    return GH_OK;
}

extern "C" int gh_polygonize_cont(const gh_grid *grid, const gh_sdb *csdb, const float *seeds, int32_t n_seeds,
                                  const gh_options *opts, gh_mesh *out, void *stream) {
    gh_sdb *s = const_cast<gh_sdb *>(csdb);
    if (!s) return fail(GH_ERR_ARG, "NULL sdb");
    gh_options o{GH_FP32, GH_TAU_DIAGONAL, -1.f, 1, 0, 0, GH_METHOD_HOP};
    if (opts) o = *opts;
    GridP g;
    int rc = check_grid(grid, &g, GH_TAU_DIAGONAL);
    if (rc) return rc;
    if ((rc = check_mesh(out))) return rc;
    if (!seeds || n_seeds < 1 || n_seeds > 65536) return fail(GH_ERR_ARG, "continuation: 1..65536 seed points needed");
    for (int i = 0; i < 3 * n_seeds; ++i)
        if (!isfinite(seeds[i])) return fail(GH_ERR_ARG, "continuation: seed point %d is not finite", i / 3);
    if (s->kind != GH_SDB_CSG) return fail(GH_ERR_UNIMPLEMENTED, "continuation runs on analytic SDBs only");
    if (o.precision != GH_FP32) return fail(GH_ERR_UNIMPLEMENTED, "continuation runs in FP32 only");
    if (wants_index(*out)) return fail(GH_ERR_UNIMPLEMENTED, "continuation: no indexed mesh output");
    int dev, nsm;
    if ((rc = ensure_device(&dev, &nsm))) return rc;
    if (dev != s->device) return fail(GH_ERR_ARG, "SDB lives on device %d, current device is %d", s->device, dev);
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->cap_seeds < n_seeds) {
        if (s->seeds) cudaFree(s->seeds);
        s->seeds = nullptr;
        s->cap_seeds = 0;
        GH_CUDA(cudaMalloc((void **)&s->seeds, sizeof(float) * 3 * n_seeds));
        s->cap_seeds = n_seeds;
    }
    const long long N2 = (long long)g.N * g.N;
    long long want_m = 8 * N2 > (1 << 16) ? 8 * N2 : (1 << 16);
    for (int attempt = 0; attempt < 4; ++attempt) {
        if ((rc = ensure_scratch(s, g.N, want_m, 2 * want_m)) || (rc = ensure_vis(s, g.N))) return rc;
        Scratch &c = s->scr;
        GH_CUDA(cudaMemcpyAsync(s->seeds, seeds, sizeof(float) * 3 * n_seeds, cudaMemcpyHostToDevice, st));
        launch_init(c, st);
        launch_cont_csg(s->d_prims, s->nprim, g, c, s->seeds, n_seeds, *out, nsm, st);
        launch_finalize(c, *out, N2, st);
        g_prof.recorded = false;
        g_prof.launches = 5;
        GH_CUDA(cudaGetLastError());
        if (!o.sync) return GH_OK;
        Counters h;
        GH_CUDA(cudaMemcpyAsync(&h, c.ctr, sizeof(h), cudaMemcpyDeviceToHost, st));
        GH_CUDA(cudaStreamSynchronize(st));
        if (h.flags & FLAG_TIMEOUT) return fail(GH_ERR_CUDA, "a bounded device wait timed out");
        if (h.flags & FLAG_MARK_OVERFLOW) {
            want_m = (long long)(h.marks + h.marks / 4 + 1024);
            continue;
        }
        if (h.flags & FLAG_NONFINITE) return fail(GH_ERR_NONFINITE, "the SDB evaluated to NaN or inf");
        if (h.tris > (unsigned long long)out->capacity_tris)
            return fail(GH_ERR_CAPACITY, "triangle buffer holds %lld, %llu needed", (long long)out->capacity_tris,
                        h.tris);
        if (out->cell_ids && h.cells > (unsigned long long)out->capacity_cells)
            return fail(GH_ERR_CAPACITY, "cell buffer holds %lld, %llu needed", (long long)out->capacity_cells,
                        h.cells);
        return GH_OK;
    }
    return fail(GH_ERR_CAPACITY, "internal scratch kept overflowing");
}

extern "C" int gh_eval(const gh_sdb *s, const float *p, int64_t n, float *out, int32_t precision, void *stream) {
    if (!s || (n > 0 && (!p || !out))) return fail(GH_ERR_ARG, "gh_eval: NULL argument");
    if (n < 0) return fail(GH_ERR_ARG, "gh_eval: n < 0");
    if (n == 0) return GH_OK;
    int dev, nsm, rc;
    if ((rc = ensure_device(&dev, &nsm))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (s->kind == GH_SDB_CSG) {
        launch_eval_points_csg(s->d_prims, s->nprim, p, n, out, st);
    } else if (precision == GH_FP32) {
        launch_eval_points_mlp_fp32(s->mlp, p, n, out, nsm, st);
    } else if (precision == GH_BF16_REFINE) {
        if (!bf16_supported(s->mlp.width) || s->mlp.n_mid > bf16_max_mid(s->mlp.width))
            return fail(GH_ERR_UNIMPLEMENTED, "no BF16 path for this width / depth");
        launch_eval_points_mlp_bf16(s->mlp, p, n, out, nsm, st);
    } else if (precision == GH_BF16_REFINE_X6) {
        if (!bf16_supported(s->mlp.width) || s->mlp.n_mid > x6_max_mid())
            return fail(GH_ERR_UNIMPLEMENTED, "no split-BF16 path for this width / depth");
        launch_eval_points_mlp_x6(s->mlp, p, n, out, nsm, st);
    } else {
        return fail(GH_ERR_ARG, "unknown precision %d", precision);
    }
    GH_CUDA(cudaGetLastError());
    return GH_OK;
}

// max |f_bf16 - f_ref| over n points p[n][3] (device), f_ref from the
// split-BF16 tensor-core evaluator (FP32-level accuracy; reading 16 of the
// design notes measures it against FP32 and FP64); d_max is a device uint.
static int bf16_gap(gh_sdb *s, const float *p, long long n, float *f32, float *f16, unsigned int *d_max, int nsm,
                    cudaStream_t st) {
    if (n <= 0) return GH_OK;
    launch_eval_points_mlp_x6(s->mlp, p, n, f32, nsm, st);
    launch_eval_points_mlp_bf16(s->mlp, p, n, f16, nsm, st);
    launch_max_abs_diff(f32, f16, n, d_max, st);
    GH_CUDA(cudaGetLastError());
    return GH_OK;
}

extern "C" int gh_sdb_calibrate(gh_sdb *s, const gh_grid *grid, int64_t n_points, uint64_t seed, float *eps_out,
                                void *stream) {
    if (!s || s->kind != GH_SDB_MLP) return fail(GH_ERR_ARG, "gh_sdb_calibrate needs a neural SDB");
    if (n_points < 0 || n_points > (1ll << 26)) return fail(GH_ERR_ARG, "n_points outside [0, 2^26]");
    if (!bf16_supported(s->mlp.width) || s->mlp.n_mid > bf16_max_mid(s->mlp.width) || s->mlp.n_mid > x6_max_mid())
        return fail(GH_ERR_UNIMPLEMENTED, "no BF16 path for this width / depth");
    GridP g;
    int rc = check_grid(grid, &g, GH_TAU_DIAGONAL);
    if (rc) return rc;
    int dev, nsm;
    if ((rc = ensure_device(&dev, &nsm))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(s->mu);
    // 1. seeded uniform points of the polygonization volume
    // 2. the lattice vertices a BF16 hopping run (no shrink) needs at a
    //    quarter of the resolution -- points next to the surface, where eps
    //    matters most (only a sample: the measured gap is the bound, the run
    //    need not find every cell)
    GridP gc = g;
    gc.N = g.N / 4 < 32 ? 32 : g.N / 4;
    gc.h = (g.h * g.N) / gc.N;
    gc.inv_h = 1.f / gc.h;
    gc.tau = (float)(sqrt(3.0) * gc.h);
    gc.eps = 0.f;
    const long long N2 = (long long)gc.N * gc.N;
    if ((rc = ensure_scratch(s, gc.N, 8 * N2 > (1 << 16) ? 8 * N2 : (1 << 16), 16 * N2 > (1 << 17) ? 16 * N2 : (1 << 17))))
        return rc;
    Scratch &c = s->scr;
    if ((rc = sync_item(s, gc, st))) return rc;
    launch_init(c, st);
    launch_hop_mlp_bf16(s->d_item, 1, s->mlp.width, nsm, 2, st);
    launch_build_lists(gc, c, st);
    Counters hc;
    GH_CUDA(cudaMemcpyAsync(&hc, c.ctr, sizeof(hc), cudaMemcpyDeviceToHost, st));
    GH_CUDA(cudaStreamSynchronize(st));
    const long long nv = (hc.flags & (FLAG_MARK_OVERFLOW | FLAG_VERT_OVERFLOW)) ? 0 : (long long)hc.verts;
    const long long nmax = n_points > nv ? n_points : nv;
    float *p = nullptr, *f32 = nullptr, *f16 = nullptr;
    unsigned int *d_max = nullptr;
    GH_CUDA(cudaMalloc((void **)&p, sizeof(float) * 3 * (nmax + 1)));
    GH_CUDA(cudaMalloc((void **)&f32, sizeof(float) * (nmax + 1)));
    GH_CUDA(cudaMalloc((void **)&f16, sizeof(float) * (nmax + 1)));
    GH_CUDA(cudaMalloc((void **)&d_max, sizeof(unsigned int)));
    GH_CUDA(cudaMemsetAsync(d_max, 0, sizeof(unsigned int), st));
    const float ext = g.h * (float)g.N;
    launch_rand_points(p, n_points, g.lo, ext, seed, st);
    rc = bf16_gap(s, p, n_points, f32, f16, d_max, nsm, st);
    if (!rc && nv > 0) {
        launch_vertex_points(gc, c, p, st);
        rc = bf16_gap(s, p, nv, f32, f16, d_max, nsm, st);
    }
    unsigned int hmax = 0;
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(&hmax, d_max, sizeof(hmax), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = fail(GH_ERR_CUDA, "calibration: %s", cudaGetErrorString(e));
    }
    cudaFree(p);
    cudaFree(f32);
    cudaFree(f16);
    cudaFree(d_max);
    if (rc) return rc;
    float gap;
    memcpy(&gap, &hmax, 4);
    if (!isfinite(gap)) return fail(GH_ERR_NONFINITE, "calibration met a non-finite value");
    s->eps = 2.f * gap;
    if (eps_out) *eps_out = s->eps;
    return GH_OK;
}

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------
struct BatchPlan {
    std::vector<int> order;          // items grouped: analytic first, then neural by (width, depth), N descending
    std::vector<std::pair<int, int>> groups;  // [begin, end) into order
    std::vector<GridP> g;            // per item (original index)
    Item *d_items = nullptr;         // device descriptors in `order`
};

static std::mutex g_graph_mu;
static std::vector<std::pair<void *, Item *>> g_graph_items;

// The launch sequence of a batch: a fixed number of launches whatever B is --
// counter reset, one persistent hopping launch per evaluator family, the
// line lists, the vertex values (one launch for the analytic items, one per
// neural family), the refinement selection and refinement, Marching Cubes
// and the status words, each step one launch over all items (the indexed
// mesh, when asked for, adds two launches per item that wants it).
static int batch_enqueue(const BatchPlan &P, int B, gh_sdb *const *sd, const gh_options &o, const gh_mesh *outs,
                         int nsm, cudaStream_t st) {
    const int tiles = o.mlp_tiles == 1 ? 1 : 2;
    int max_N = 2, max_prims = 1;
    bool any_csg = false, any_mlp = false;
    for (int b = 0; b < B; ++b) {
        max_N = P.g[b].N > max_N ? P.g[b].N : max_N;
        if (sd[b]->kind == GH_SDB_CSG) {
            any_csg = true;
            max_prims = sd[b]->nprim > max_prims ? sd[b]->nprim : max_prims;
        } else {
            any_mlp = true;
        }
    }
    long long launches = 1 + 8 + 1 + 1;  // counters, lists, Marching Cubes, status words
    launch_init_b(P.d_items, B, st);
    for (auto &gr : P.groups) {
        ++launches;
        const gh_sdb *first = sd[P.order[gr.first]];
        const Item *di = P.d_items + gr.first;
        const int n = gr.second - gr.first;
        if (first->kind == GH_SDB_CSG) {
            int mx = 1;
            for (int q = gr.first; q < gr.second; ++q) mx = sd[P.order[q]]->nprim > mx ? sd[P.order[q]]->nprim : mx;
            launch_hop_csg(di, n, mx, nsm, o.ray_block, st);
        } else if (o.precision == GH_FP32) {
            launch_hop_mlp_fp32(di, n, first->mlp.width, nsm, st);
        } else {
            launch_hop_mlp_bf16(di, n, first->mlp.width, nsm, tiles, st);
        }
    }
    launch_build_lists_b(P.d_items, B, max_N, nsm, st);
    if (any_csg) {
        launch_eval_vertices_csg_b(P.d_items, B, max_prims, nsm, st);
        ++launches;
    }
    for (auto &gr : P.groups) {
        const gh_sdb *first = sd[P.order[gr.first]];
        if (first->kind == GH_SDB_CSG) continue;
        const Item *di = P.d_items + gr.first;
        const int n = gr.second - gr.first;
        ++launches;
        if (o.precision == GH_FP32) launch_eval_vertices_mlp_fp32(di, n, first->mlp.width, nsm, false, st);
        else launch_eval_vertices_mlp_bf16(di, n, first->mlp.width, nsm, tiles, st);
    }
    if (any_mlp && o.precision != GH_FP32) {
        launch_refine_select_b(P.d_items, B, nsm, st);
        launches += 3;
        for (auto &gr : P.groups) {
            const gh_sdb *first = sd[P.order[gr.first]];
            if (first->kind == GH_SDB_CSG) continue;
            const Item *di = P.d_items + gr.first;
            const int n = gr.second - gr.first;
            ++launches;
            if (o.precision == GH_BF16_REFINE_X6) launch_refine_mlp_x6(di, n, first->mlp.width, nsm, st);
            else launch_eval_vertices_mlp_fp32(di, n, first->mlp.width, nsm, true, st);
        }
    }
    launch_mc_b(P.d_items, B, nsm, st);
    for (int b = 0; b < B; ++b)
        if (wants_index(outs[b])) {
            launch_index_mesh(P.g[b], sd[b]->scr, outs[b], nsm, st);
            launches += 5;  // at most
        }
    launch_finalize_b(P.d_items, B, st);
    g_prof.recorded = false;
    g_prof.launches = launches;
    GH_CUDA(cudaGetLastError());
    return GH_OK;
}

extern "C" int gh_polygonize_batch(int B, const gh_grid *grids, const gh_sdb *const *sdbs, const gh_options *opts,
                                   gh_mesh *outs, void *stream, void **graph) {
    if (B < 1 || !grids || !sdbs || !outs) return fail(GH_ERR_ARG, "gh_polygonize_batch: empty or NULL arguments");
    gh_options o{GH_FP32, GH_TAU_DIAGONAL, -1.f, 1, 0, 0, GH_METHOD_HOP};
    if (opts) o = *opts;
    if (o.precision != GH_FP32 && o.precision != GH_BF16_REFINE && o.precision != GH_BF16_REFINE_X6)
        return fail(GH_ERR_ARG, "unknown precision %d", o.precision);
    if (o.method != GH_METHOD_HOP) return fail(GH_ERR_UNIMPLEMENTED, "batches run grid hopping only");
    int dev, nsm, rc;
    if ((rc = ensure_device(&dev, &nsm))) return rc;
    std::vector<gh_sdb *> sd(B);
    BatchPlan P;
    P.g.resize(B);
    for (int b = 0; b < B; ++b) {
        sd[b] = const_cast<gh_sdb *>(sdbs[b]);
        if (!sd[b]) return fail(GH_ERR_ARG, "item %d: NULL sdb", b);
        for (int q = 0; q < b; ++q)
            if (sd[q] == sd[b]) return fail(GH_ERR_ARG, "items %d and %d share one SDB object", q, b);
        if (sd[b]->device != dev) return fail(GH_ERR_ARG, "item %d: SDB on another device", b);
        if ((rc = check_grid(&grids[b], &P.g[b], o.tau_mode))) return rc;
        if ((rc = check_mesh(&outs[b]))) return rc;
        if (sd[b]->kind == GH_SDB_MLP && o.precision != GH_FP32) {
            if (sd[b]->mlp.n_mid > bf16_max_mid(sd[b]->mlp.width))
                return fail(GH_ERR_UNIMPLEMENTED, "item %d: BF16 path supports at most %d hidden layers", b,
                            bf16_max_mid(sd[b]->mlp.width));
            const float eps = o.eps >= 0.f ? o.eps : sd[b]->eps;
            if (!(eps >= 0.f)) return fail(GH_ERR_ARG, "item %d: BF16 needs eps (calibrate the SDB)", b);
            P.g[b].eps = eps;
        }
    }
    // groups: analytic items, then neural items by (width, depth); N descending inside a group
    std::vector<int> idx(B);
    for (int b = 0; b < B; ++b) idx[b] = b;
    auto key = [&](int b) {
        const gh_sdb *x = sd[b];
        return x->kind == GH_SDB_CSG ? 0 : 1 + x->mlp.width * 64 + x->mlp.n_mid;
    };
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
        if (key(a) != key(b)) return key(a) < key(b);
        return P.g[a].N > P.g[b].N;
    });
    P.order = idx;
    for (int q = 0; q < B;) {
        int e = q;
        while (e < B && key(idx[e]) == key(idx[q])) ++e;
        P.groups.push_back({q, e});
        q = e;
    }
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<std::unique_lock<std::mutex>> locks;
    for (int b = 0; b < B; ++b) locks.emplace_back(sd[b]->mu);
    std::vector<long long> want_m(B), want_v(B);
    for (int b = 0; b < B; ++b) {
        const long long N2 = (long long)P.g[b].N * P.g[b].N;
        want_m[b] = 8 * N2 > (1 << 16) ? 8 * N2 : (1 << 16);
        want_v[b] = 2 * want_m[b];
    }
    Item *d_items = nullptr;
    GH_CUDA(cudaMalloc((void **)&d_items, sizeof(Item) * B));
    P.d_items = d_items;
    std::vector<Item> h_items(B);
    const bool sync = o.sync || graph;
    for (int attempt = 0; attempt < 4; ++attempt) {
        for (int b = 0; b < B; ++b)
            if ((rc = ensure_scratch(sd[b], P.g[b].N, want_m[b], want_v[b])) ||
                (wants_index(outs[b]) && (rc = ensure_index(sd[b])))) {
                cudaFree(d_items);
                return rc;
            }
        for (int q = 0; q < B; ++q) {
            h_items[q] = make_item(sd[P.order[q]], P.g[P.order[q]]);
            h_items[q].out = outs[P.order[q]];
        }
        GH_CUDA(cudaMemcpyAsync(d_items, h_items.data(), sizeof(Item) * B, cudaMemcpyHostToDevice, st));
        if ((rc = batch_enqueue(P, B, sd.data(), o, outs, nsm, st))) {
            cudaFree(d_items);
            return rc;
        }
        if (!sync) break;  // asynchronous: d_items must outlive the work; keep it with the last batch
        GH_CUDA(cudaStreamSynchronize(st));
        bool grow = false;
        for (int b = 0; b < B; ++b) {
            Counters c;
            GH_CUDA(cudaMemcpy(&c, sd[b]->scr.ctr, sizeof(c), cudaMemcpyDeviceToHost));
            if (c.flags & FLAG_TIMEOUT) {
                cudaFree(d_items);
                return fail(GH_ERR_CUDA, "item %d: a bounded device wait timed out", b);
            }
            if (c.flags & (FLAG_MARK_OVERFLOW | FLAG_VERT_OVERFLOW)) {
                if (c.flags & FLAG_MARK_OVERFLOW) want_m[b] = (long long)(c.marks + c.marks / 4 + 1024);
                want_v[b] = (c.flags & FLAG_VERT_OVERFLOW) ? (long long)(c.verts + c.verts / 4 + 1024) : 2 * want_m[b];
                if (want_v[b] < 2 * want_m[b]) want_v[b] = 2 * want_m[b];
                grow = true;
            }
        }
        if (grow) continue;
        rc = GH_OK;
        for (int b = 0; b < B && rc == GH_OK; ++b) {
            Counters c;
            GH_CUDA(cudaMemcpy(&c, sd[b]->scr.ctr, sizeof(c), cudaMemcpyDeviceToHost));
            if (c.flags & FLAG_NONFINITE) rc = fail(GH_ERR_NONFINITE, "item %d: NaN or inf", b);
            else if (c.tris > (unsigned long long)outs[b].capacity_tris)
                rc = fail(GH_ERR_CAPACITY, "item %d: triangle buffer holds %lld, %llu needed", b,
                          (long long)outs[b].capacity_tris, c.tris);
            else if (outs[b].cell_ids && c.cells > (unsigned long long)outs[b].capacity_cells)
                rc = fail(GH_ERR_CAPACITY, "item %d: cell buffer too small", b);
            else if (c.flags & FLAG_INDEX_MISS)
                rc = fail(GH_ERR_CUDA, "item %d: indexed output: a triangle edge was not listed", b);
            else if (outs[b].vert_xyz && c.mesh_verts > (unsigned long long)outs[b].capacity_verts)
                rc = fail(GH_ERR_CAPACITY, "item %d: vertex buffer holds %lld, %llu needed", b,
                          (long long)outs[b].capacity_verts, c.mesh_verts);
        }
        if (rc || !graph) {
            cudaFree(d_items);
            return rc;
        }
        // capture the same sequence into a graph bound to these buffers, on a
        // private stream (the legacy default stream can not be captured)
        cudaGraph_t gr = nullptr;
        cudaStream_t cs = nullptr;
        GH_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaError_t ec = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        int erc = GH_OK;
        if (ec == cudaSuccess) {
            erc = batch_enqueue(P, B, sd.data(), o, outs, nsm, cs);
            ec = cudaStreamEndCapture(cs, &gr);
        }
        cudaStreamDestroy(cs);
        if (erc || ec != cudaSuccess) {
            if (gr) cudaGraphDestroy(gr);
            cudaFree(d_items);
            return erc ? erc : fail(GH_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ec));
        }
        cudaGraphExec_t ex = nullptr;
        const cudaError_t ei = cudaGraphInstantiate(&ex, gr, 0);
        cudaGraphDestroy(gr);
        if (ei != cudaSuccess) {
            cudaFree(d_items);
            return fail(GH_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ei));
        }
        {
            std::lock_guard<std::mutex> lk(g_graph_mu);
            g_graph_items.push_back({(void *)ex, d_items});
        }
        *graph = (void *)ex;
        return GH_OK;
    }
    if (!sync) {
        // the descriptors must live until the stream has consumed them
        std::lock_guard<std::mutex> lk(g_graph_mu);
        g_graph_items.push_back({nullptr, d_items});
        return GH_OK;
    }
    cudaFree(d_items);
    return fail(GH_ERR_CAPACITY, "internal scratch kept overflowing");
}

extern "C" int gh_batch_graph_launch(void *graph, void *stream) {
    if (!graph) return fail(GH_ERR_ARG, "gh_batch_graph_launch: NULL graph");
    GH_CUDA(cudaGraphLaunch((cudaGraphExec_t)graph, (cudaStream_t)stream));
    return GH_OK;
}

extern "C" int gh_batch_graph_free(void *graph) {
    if (!graph) return GH_OK;
    Item *items = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_graph_mu);
        for (size_t i = 0; i < g_graph_items.size(); ++i)
            if (g_graph_items[i].first == graph) {
                items = g_graph_items[i].second;
                g_graph_items.erase(g_graph_items.begin() + i);
                break;
            }
    }
    GH_CUDA(cudaGraphExecDestroy((cudaGraphExec_t)graph));
    if (items) cudaFree(items);
    return GH_OK;
}

extern "C" int gh_backward(const gh_sdb *cs, const float *verts, const float *dL_dv, int64_t V, float *dL_dtheta,
                           void *stream) {
    gh_sdb *s = const_cast<gh_sdb *>(cs);
    if (!s) return fail(GH_ERR_ARG, "gh_backward: NULL sdb");
    if (V < 0 || V > (1ll << 31) - 1) return fail(GH_ERR_ARG, "gh_backward: V = %lld out of range", (long long)V);
    if (!dL_dtheta || (V > 0 && (!verts || !dL_dv))) return fail(GH_ERR_ARG, "gh_backward: NULL pointer");
    int dev, nsm, rc;
    if ((rc = ensure_device(&dev, &nsm))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (s->kind == GH_SDB_CSG) {
        std::lock_guard<std::mutex> lk(s->mu);
        const size_t need = (size_t)7 * (size_t)(V > 0 ? V : 1);
        if (s->adj_floats < need) {
            if (s->adj) cudaFree(s->adj);
            s->adj = nullptr;
            s->adj_floats = 0;
            GH_CUDA(cudaMalloc((void **)&s->adj, sizeof(float) * need));
            s->adj_floats = need;
        }
        int *act = reinterpret_cast<int *>(s->adj);
        float *contrib = s->adj + (V > 0 ? V : 1);
        csg_adjoint(s->d_prims, s->nprim, verts, dL_dv, (int)V, act, contrib, dL_dtheta, st);
        GH_CUDA(cudaGetLastError());
        return GH_OK;
    }
    if (V == 0) {
        GH_CUDA(cudaMemsetAsync(dL_dtheta, 0, sizeof(float) * s->nparam, st));
        return GH_OK;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    const int W = s->mlp.width, L = s->mlp.n_mid, S = 76;  // 2 x 76 weight-gradient tiles: one per SM
    // vertices per chunk: the stored activations and deltas of a chunk take
    // 2 (L + 1) W floats per vertex (1.6 GB at W = 256, L = 5)
    constexpr int VCHUNK = GH_ADJOINT_CHUNK;
    const size_t need = adjoint_buffer_floats(W, L, VCHUNK, S);
    if (s->adj_floats < need) {
        if (s->adj) cudaFree(s->adj);
        s->adj = nullptr;
        s->adj_floats = 0;
        GH_CUDA(cudaMalloc((void **)&s->adj, sizeof(float) * need));
        s->adj_floats = need;
    }
    AdjBuffers b;
    b.VC = VCHUNK;
    b.splits = S;
    b.nsm = nsm;
    b.Z = s->adj;
    b.D = b.Z + (size_t)(L + 1) * b.VC * W;
    b.s = b.D + (size_t)(L + 1) * b.VC * W;
    b.part = b.s + b.VC;
    b.ones = b.part + (size_t)S * W * W;
    b.mbits = reinterpret_cast<uint32_t *>(b.ones + b.VC);
    adjoint_fill_ones(b.ones, b.VC, st);
    for (long long v0 = 0; v0 < V; v0 += b.VC) {
        const int n = (int)((V - v0) < b.VC ? (V - v0) : b.VC);
        adjoint_chunk(s->mlp, verts + 3 * v0, dL_dv + 3 * v0, n, dL_dtheta, v0 > 0, b, st);
    }
    GH_CUDA(cudaGetLastError());
    return GH_OK;
}

// ---------------------------------------------------------------------------
// No-allocation variant (analytic scenes): the scratch of the pipeline lives
// in one file-scope device array instead of per-SDB cudaMalloc'd buffers.
// Host code must not use the array's name as an address (it is a host-side
// stand-in); the device address is looked up once per device below.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[GH_NOALLOC_SCRATCH_BYTES];
static __device__ Item g_noalloc_item;  // descriptor of the call (static, like the scratch)
static void *g_noalloc_item_addr[64];
static void *g_noalloc_addr[64];
static std::mutex g_noalloc_mu;

static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

extern "C" int gh_polygonize_csg_noalloc(const gh_grid *grid, const gh_csg_prim *prims, int32_t n_prim,
                                         int32_t tau_mode, gh_mesh *out, void *stream) {
    GridP g;
    int rc = check_grid(grid, &g, tau_mode);
    if (rc) return rc;
    if (g.N > GH_NOALLOC_MAX_N)
        return fail(GH_ERR_ARG, "gh_polygonize_csg_noalloc: N = %d exceeds GH_NOALLOC_MAX_N = %d", g.N,
                    GH_NOALLOC_MAX_N);
    if (!prims) return fail(GH_ERR_ARG, "gh_polygonize_csg_noalloc: NULL prims");
    if (n_prim < 1 || n_prim > GH_MAX_PRIMS)
        return fail(GH_ERR_ARG, "gh_polygonize_csg_noalloc: n_prim = %d outside [1, %d]", n_prim, GH_MAX_PRIMS);
    if ((rc = check_mesh(out))) return rc;
    if (wants_index(*out)) return fail(GH_ERR_UNIMPLEMENTED, "gh_polygonize_csg_noalloc: no indexed mesh output");
    int dev, nsm;
    if ((rc = ensure_device(&dev, &nsm))) return rc;
    constexpr int NDEV = (int)(sizeof(g_noalloc_addr) / sizeof(g_noalloc_addr[0]));
    if (dev < 0 || dev >= NDEV)
        return fail(GH_ERR_DEVICE, "gh_polygonize_csg_noalloc: device %d beyond the %d this library tracks", dev, NDEV);
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return fail(GH_ERR_CUDA, "cudaGetSymbolAddress(no-allocation scratch): %s", cudaGetErrorString(e));
            g_noalloc_addr[dev] = p;
            void *pi = nullptr;
            const cudaError_t e2 = cudaGetSymbolAddress(&pi, g_noalloc_item);
            if (e2 != cudaSuccess || !pi)
                return fail(GH_ERR_CUDA, "cudaGetSymbolAddress(no-allocation descriptor): %s", cudaGetErrorString(e2));
            g_noalloc_item_addr[dev] = pi;
        }
        base = g_noalloc_addr[dev];
    }
    Item *ditem = (Item *)g_noalloc_item_addr[dev];
    // carve the array for the largest grid it accepts
    const size_t NN = GH_NOALLOC_MAX_N, ncols = NN * NN, nlines = (NN + 1) * (NN + 1);
    char *q = (char *)base;
    size_t off = 0;
    Scratch c{};
    c.ctr = (Counters *)(q + off);
    off += up256(sizeof(Counters));
    Prim *staged = (Prim *)(q + off);  // the caller's records with their bounding radii
    off += up256(sizeof(Prim) * GH_MAX_PRIMS);
    c.colcount = (uint32_t *)(q + off);
    off += up256(4 * ncols);
    c.coloff = (uint32_t *)(q + off);
    off += up256(4 * (ncols + 1));
    c.linecount = (uint32_t *)(q + off);
    off += up256(4 * nlines);
    c.lineoff = (uint32_t *)(q + off);
    off += up256(4 * (nlines + 1));
    c.blocksum = (uint32_t *)(q + off);
    off += up256(4 * 4096);
    const size_t per = 2 * 8 + 2 * (8 + 4);  // marks raw + grouped, two vertices (key + value) per mark
    const size_t M = ((GH_NOALLOC_SCRATCH_BYTES - off - 4 * 256) / per) & ~(size_t)255;
    c.marks_raw = (unsigned long long *)(q + off);
    off += up256(8 * M);
    c.marks_csr = (unsigned long long *)(q + off);
    off += up256(8 * M);
    c.vkey = (unsigned long long *)(q + off);
    off += up256(8 * 2 * M);
    c.vval = (float *)(q + off);
    off += up256(4 * 2 * M);
    c.cap_marks = (long long)M;
    c.cap_verts = (long long)(2 * M);
    if (off > GH_NOALLOC_SCRATCH_BYTES) return fail(GH_ERR_CUDA, "no-allocation scratch layout overflows");
    cudaStream_t st = (cudaStream_t)stream;
    const Prim *dp = staged;
    Item hitem{};
    hitem.g = g;
    hitem.s = c;
    hitem.prims = dp;
    hitem.nprim = n_prim;
    hitem.kind = GH_SDB_CSG;
    GH_CUDA(cudaMemcpyAsync(ditem, &hitem, sizeof(Item), cudaMemcpyHostToDevice, st));
    launch_init(c, st);  // clears the counters left by the previous call
    launch_stage_prims(reinterpret_cast<const Prim *>(prims), staged, n_prim, st);
    launch_hop_csg(ditem, 1, n_prim, nsm, 256, st);
    launch_build_lists(g, c, st);
    launch_eval_vertices_csg(dp, n_prim, g, c, nsm, st);
    launch_mc(g, c, *out, nsm, st);
    launch_finalize(c, *out, (long long)g.N * g.N, st);
    GH_CUDA(cudaGetLastError());
    Counters h;
    GH_CUDA(cudaMemcpyAsync(&h, c.ctr, sizeof(h), cudaMemcpyDeviceToHost, st));
    GH_CUDA(cudaStreamSynchronize(st));
    if (h.flags & FLAG_MARK_OVERFLOW)
        return fail(GH_ERR_CAPACITY, "scene marks %llu cells; the no-allocation scratch holds %lld", h.marks,
                    c.cap_marks);
    if (h.flags & FLAG_VERT_OVERFLOW)
        return fail(GH_ERR_CAPACITY, "scene needs %llu lattice vertices; the no-allocation scratch holds %lld",
                    h.verts, c.cap_verts);
    if (h.flags & FLAG_NONFINITE) return fail(GH_ERR_NONFINITE, "the SDB evaluated to NaN or inf");
    if (h.tris > (unsigned long long)out->capacity_tris)
        return fail(GH_ERR_CAPACITY, "triangle buffer holds %lld, %llu needed", (long long)out->capacity_tris, h.tris);
    if (out->cell_ids && h.cells > (unsigned long long)out->capacity_cells)
        return fail(GH_ERR_CAPACITY, "cell buffer holds %lld, %llu needed", (long long)out->capacity_cells, h.cells);
    return GH_OK;
}
