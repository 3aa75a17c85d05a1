/*
 * Grid-hopping polygonizer -- plain FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  The product path never calls, links or loads
 * this file: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or constant
 * generator with the CUDA library; its inputs are plain arrays produced by
 * the seeded input generators.
 *
 * Paper: N. Markus, M. Suznjevic, "Theoretical and Empirical Analysis of a
 * Fast Algorithm for Extracting Polygons from Signed Distance Bounds".
 *
 *   Sec. 1     signed distance bound (SDB): |f(x)| never exceeds the distance
 *              from x to the zero set; negative inside.
 *   Sec. 3     grid of N^3 cells over an axis-aligned cube (Eq. 1), N^2 rays
 *              along +z (Eq. 2), the sphere-tracing iteration (Eq. 3), the
 *              polygonization distance (Eq. 4) and Algorithm 1.
 *   Sec. 4.1   plane distance (Eq. 5); Sec. 4.2 box distance (Eq. 6) and the
 *              exact box distance; Sec. 4.3 union of shapes by min.
 *   Sec. 2     enumeration: Marching Cubes on every one of the N^3 cells.
 *   Sec. 5     every method compared there yields the identical mesh (the
 *              invariant the tests check); Sec. 5.2 the neural SDB (Eq. 7)
 *              shrunk by lambda.
 *
 * Conventions (the paper's unit cube generalised to [lo, lo + N h]^3):
 *   cell (i,j,k) = [lo+ih, lo+(i+1)h] x ... ; its centre lo + (i+1/2)h ...
 *   lattice vertex (a,b,c) = lo + (a,b,c) h, 0 <= a,b,c <= N.
 *   corner bit b of a cell sits at offset (b&1, b>>1&1, b>>2&1).
 *   inside <=> f < 0, so f == 0 counts as outside.
 *   case = sum over corners of [f_b < 0] << b.
 *   edge e = 4*axis + (u + 2v), (u,v) = the offsets of its lower endpoint on
 *   the other two axes taken in increasing axis order.
 *   edge key = axis*(N+1)^3 + (a + (N+1)(b + (N+1)c)), (a,b,c) = the lower
 *   endpoint of the edge on the lattice.
 *   vertex on a crossing edge: t = fA/(fA - fB) from the lower endpoint A.
 *   triangles are oriented so that (v1-v0)x(v2-v0) points towards f > 0.
 *
 * Everything is double precision.  OpenMP parallelises independent columns
 * or cells; per-item arithmetic is not reordered.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* SDB descriptions                                                          */
/* ------------------------------------------------------------------------ */

enum { OR_SPHERE = 0, OR_TORUS = 1, OR_BOX = 2, OR_CAPSULE = 3, OR_CYLINDER = 4, OR_HEXPRISM = 5, OR_CONE = 6 };
enum { OR_UNION = 0, OR_SUBTRACT = 1, OR_INTERSECT = 2 };
#define OR_PRIM_STRIDE 17 /* type, op, c[3], p[3], rot[9] */

typedef struct {
    int kind; /* 0 = CSG, 1 = MLP */
    /* CSG: a left fold over primitives, f = op_n(...op_1(d_0, d_1)..., d_n) */
    int nprim;
    double *prim;
    /* MLP: g = w_out . relu(W_m ... relu(W_0 p + b_0) ...) + b_out */
    int width, nmid;
    double *W0, *b0;   /* [width,3], [width] */
    double **Wm, **bm; /* nmid x [width,width], nmid x [width] */
    double *wout, bout;
    double r0, alpha, beta, lam; /* f = (rad |p| - r0 + alpha g) / beta / lam */
    double rad;                  /* 1, or 0 for a network without the radial term */
    /* lattice: trilinear interpolation of given values at the lattice points
     * of a grid (a test device for Marching Cubes, not an SDB in general) */
    int ln;
    double llo[3], lh, *lval;
} osdb;

/* Sphere: distance to a ball's boundary (Sec. 5.1 primitive list). */
static double d_sphere(const double *q, const double *prm) {
    return sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]) - prm[0];
}

/* Torus around the local y axis, major radius R, minor radius r. */
static double d_torus(const double *q, const double *prm) {
    double a = sqrt(q[0] * q[0] + q[2] * q[2]) - prm[0];
    return sqrt(a * a + q[1] * q[1]) - prm[1];
}

/* Exact distance to a box with half sizes prm (Sec. 4.2, the exact variant
 * of the max-of-six-planes bound of Eq. 6). */
static double d_box(const double *q, const double *prm) {
    double e[3], out2 = 0.0, inmax = -INFINITY;
    for (int a = 0; a < 3; ++a) {
        e[a] = fabs(q[a]) - prm[a];
        if (e[a] > 0) out2 += e[a] * e[a];
        if (e[a] > inmax) inmax = e[a];
    }
    return sqrt(out2) + (inmax < 0 ? inmax : 0.0);
}

/* Capsule: the points within r of the segment from (0,-H,0) to (0,H,0). */
static double d_capsule(const double *q, const double *prm) {
    double y = q[1] < -prm[0] ? -prm[0] : (q[1] > prm[0] ? prm[0] : q[1]);
    double v[3] = {q[0], q[1] - y, q[2]};
    return sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) - prm[1];
}

/* Capped cylinder around the local y axis: radius r, half height H.  In the
 * (radius, height) half-plane the solid is the rectangle [0,r] x [-H,H]. */
static double d_cylinder(const double *q, const double *prm) {
    double e0 = sqrt(q[0] * q[0] + q[2] * q[2]) - prm[0], e1 = fabs(q[1]) - prm[1];
    double o0 = e0 > 0 ? e0 : 0.0, o1 = e1 > 0 ? e1 : 0.0;
    double in = e0 > e1 ? e0 : e1;
    return sqrt(o0 * o0 + o1 * o1) + (in < 0 ? in : 0.0);
}

/* 2-D signed distance to the regular hexagon of apothem a whose edges face
 * the directions 0, 60, ..., 300 degrees: by symmetry fold into the wedge of
 * angles [-30, 30] degrees, where the nearest edge is x = a, |z| <= a/sqrt(3). */
static double d_hexagon2(double x, double z, double a) {
    x = fabs(x);
    z = fabs(z);
    const double mx = -0.5, mz = sqrt(3.0) / 2; /* normal of the 30-degree mirror */
    double dot = x * mx + z * mz;
    if (dot > 0) {
        x -= 2 * dot * mx;
        z -= 2 * dot * mz;
    }
    double lim = a / sqrt(3.0), zc = z < -lim ? -lim : (z > lim ? lim : z);
    double v0 = x - a, v1 = z - zc, n = sqrt(v0 * v0 + v1 * v1);
    return v0 < 0 ? -n : n;
}

/* Hexagonal prism: the hexagon (apothem a) in the local xz-plane, extruded
 * over |y| <= H. */
static double d_hexprism(const double *q, const double *prm) {
    double e0 = d_hexagon2(q[0], q[2], prm[0]), e1 = fabs(q[1]) - prm[1];
    double o0 = e0 > 0 ? e0 : 0.0, o1 = e1 > 0 ? e1 : 0.0;
    double in = e0 > e1 ? e0 : e1;
    return sqrt(o0 * o0 + o1 * o1) + (in < 0 ? in : 0.0);
}

/* Solid cone around the local y axis: base disc of radius R at y = -H, apex at
 * y = +H.  In the (radius rho, height y) half-plane the solid is the triangle
 * (0,-H), (R,-H), (0,H); its boundary there is the base segment and the slant
 * segment (the axis is inside the solid of revolution). */
static double d_cone(const double *q, const double *prm) {
    double R = prm[0], H = prm[1];
    double rho = sqrt(q[0] * q[0] + q[2] * q[2]), y = q[1];
    double bs = rho < 0 ? 0 : (rho > R ? R : rho);
    double b0 = rho - bs, b1 = y + H, db = sqrt(b0 * b0 + b1 * b1);
    double e0 = -R, e1 = 2 * H;
    double t = ((rho - R) * e0 + (y + H) * e1) / (e0 * e0 + e1 * e1);
    t = t < 0 ? 0 : (t > 1 ? 1 : t);
    double s0 = rho - (R + t * e0), s1 = y - (-H + t * e1), ds = sqrt(s0 * s0 + s1 * s1);
    double d = db < ds ? db : ds;
    int inside = y > -H && y < H && rho * 2 * H < R * (H - y);
    return inside ? -d : d;
}

static double prim_eval(const double *pr, const double *p) {
    const double *c = pr + 2, *prm = pr + 5, *R = pr + 8;
    double d[3] = {p[0] - c[0], p[1] - c[1], p[2] - c[2]};
    double q[3];
    for (int r = 0; r < 3; ++r) q[r] = R[3 * r] * d[0] + R[3 * r + 1] * d[1] + R[3 * r + 2] * d[2];
    switch ((int)pr[0]) {
    case OR_SPHERE: return d_sphere(q, prm);
    case OR_TORUS: return d_torus(q, prm);
    case OR_CAPSULE: return d_capsule(q, prm);
    case OR_CYLINDER: return d_cylinder(q, prm);
    case OR_HEXPRISM: return d_hexprism(q, prm);
    case OR_CONE: return d_cone(q, prm);
    default: return d_box(q, prm);
    }
}

/* CSG: union by min (Sec. 4.3), subtraction by max(f, -d), intersection by
 * max(f, d).  All three keep a 1-Lipschitz function 1-Lipschitz. */
static double csg_eval(const osdb *s, const double *p) {
    double f = prim_eval(s->prim, p);
    for (int n = 1; n < s->nprim; ++n) {
        const double *pr = s->prim + (size_t)n * OR_PRIM_STRIDE;
        double d = prim_eval(pr, p);
        switch ((int)pr[1]) {
        case OR_UNION: f = fmin(f, d); break;
        case OR_SUBTRACT: f = fmax(f, -d); break;
        default: f = fmax(f, d); break;
        }
    }
    return f;
}

/* Neural SDB (Sec. 5.2, Eq. 7): a ReLU MLP g, used as
 * f(p) = (|p| - r0 + alpha g(p)) / beta, then shrunk by lambda; a network
 * given without the radial term (rad = 0, the paper's own networks of
 * Sec. 5.2, where the SDB is the network's output divided by lambda) drops
 * |p|.
 * If acts != NULL the pre-activations z_l of every hidden layer are stored
 * there, layer after layer, (1 + nmid) * width doubles. */
static double mlp_g(const osdb *s, const double *p, double *acts) {
    int W = s->width;
    double *a = (double *)malloc(sizeof(double) * 2 * W), *b = a + W;
    for (int o = 0; o < W; ++o) {
        double z = s->b0[o] + s->W0[3 * o] * p[0] + s->W0[3 * o + 1] * p[1] + s->W0[3 * o + 2] * p[2];
        if (acts) acts[o] = z;
        a[o] = z > 0 ? z : 0.0;
    }
    for (int l = 0; l < s->nmid; ++l) {
        const double *Wl = s->Wm[l], *bl = s->bm[l];
        for (int o = 0; o < W; ++o) {
            double z = bl[o];
            for (int i = 0; i < W; ++i) z += Wl[(size_t)o * W + i] * a[i];
            if (acts) acts[(size_t)(l + 1) * W + o] = z;
            b[o] = z > 0 ? z : 0.0;
        }
        double *t = a; a = b; b = t;
    }
    double g = s->bout;
    for (int i = 0; i < W; ++i) g += s->wout[i] * a[i];
    free(a < b ? a : b);
    return g;
}

static double lattice_eval(const osdb *s, const double *p) {
    int n = s->ln, i0[3];
    double w[3];
    for (int a = 0; a < 3; ++a) {
        double u = (p[a] - s->llo[a]) / s->lh, r = floor(u + 0.5);
        if (fabs(u - r) < 1e-9) u = r; /* lattice points read their value exactly */
        if (u < 0) u = 0;
        if (u > n) u = n;
        i0[a] = (int)floor(u);
        if (i0[a] >= n) i0[a] = n - 1;
        w[a] = u - i0[a];
    }
    double f = 0;
    for (int b = 0; b < 8; ++b) {
        int x = b & 1, y = (b >> 1) & 1, z = (b >> 2) & 1;
        double wt = (x ? w[0] : 1 - w[0]) * (y ? w[1] : 1 - w[1]) * (z ? w[2] : 1 - w[2]);
        if (wt == 0) continue;
        size_t idx = (size_t)(i0[0] + x) + (size_t)(n + 1) * ((size_t)(i0[1] + y) + (size_t)(n + 1) * (i0[2] + z));
        f += wt * s->lval[idx];
    }
    return f;
}

static double sdb_eval(const osdb *s, const double *p) {
    if (s->kind == 0) return csg_eval(s, p);
    if (s->kind == 2) return lattice_eval(s, p);
    double r = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    return (s->rad * r - s->r0 + s->alpha * mlp_g(s, p, NULL)) / s->beta / s->lam;
}

void *or_csg_new(int nprim, const double *prims) {
    if (nprim < 1) return NULL;
    osdb *s = (osdb *)calloc(1, sizeof(osdb));
    s->kind = 0;
    s->nprim = nprim;
    s->prim = (double *)malloc(sizeof(double) * OR_PRIM_STRIDE * nprim);
    memcpy(s->prim, prims, sizeof(double) * OR_PRIM_STRIDE * nprim);
    return s;
}

/* params: W0[W*3] b0[W] { Wl[W*W] bl[W] } x nmid  wout[W] bout */
void *or_mlp_new(int width, int nmid, const double *params, double r0, double alpha, double beta,
                 double lam, double rad) {
    osdb *s = (osdb *)calloc(1, sizeof(osdb));
    int W = width;
    size_t n = (size_t)W * 3 + W + (size_t)nmid * ((size_t)W * W + W) + W + 1;
    double *buf = (double *)malloc(sizeof(double) * n);
    memcpy(buf, params, sizeof(double) * n);
    s->kind = 1;
    s->width = W;
    s->nmid = nmid;
    s->W0 = buf;
    s->b0 = buf + 3 * W;
    double *q = s->b0 + W;
    s->Wm = (double **)malloc(sizeof(double *) * (nmid > 0 ? nmid : 1));
    s->bm = (double **)malloc(sizeof(double *) * (nmid > 0 ? nmid : 1));
    for (int l = 0; l < nmid; ++l) {
        s->Wm[l] = q;
        q += (size_t)W * W;
        s->bm[l] = q;
        q += W;
    }
    s->wout = q;
    s->bout = q[W];
    s->r0 = r0;
    s->alpha = alpha;
    s->beta = beta;
    s->lam = lam;
    s->rad = rad;
    s->prim = buf; /* owner of the parameter block */
    return s;
}

/* values[(N+1)^3], index a + (N+1)(b + (N+1)c) */
void *or_lattice_new(int n, const double *lo, double h, const double *values) {
    osdb *s = (osdb *)calloc(1, sizeof(osdb));
    size_t m = (size_t)(n + 1) * (n + 1) * (n + 1);
    s->kind = 2;
    s->ln = n;
    s->lh = h;
    memcpy(s->llo, lo, sizeof(double) * 3);
    s->lval = (double *)malloc(sizeof(double) * m);
    memcpy(s->lval, values, sizeof(double) * m);
    s->prim = s->lval;
    return s;
}

void or_sdb_free(void *h) {
    osdb *s = (osdb *)h;
    if (!s) return;
    free(s->prim);
    free(s->Wm);
    free(s->bm);
    free(s);
}

void or_eval(const void *h, int64_t n, const double *p, double *out) {
    const osdb *s = (const osdb *)h;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) out[i] = sdb_eval(s, p + 3 * i);
}

/* ------------------------------------------------------------------------ */
/* Marching Cubes table, generated from a per-face rule                     */
/* ------------------------------------------------------------------------ */
/*
 * The paper polygonizes each cell with Marching Cubes (Sec. 3, Sec. 5) but
 * prints no table, so the oracle derives its own:
 *   1. the crossing edges of a case are the edges whose endpoints differ in
 *      sign;
 *   2. on every cube face the crossing edges are joined in pairs by
 *      segments: two crossings give one segment; four crossings (an
 *      ambiguous face, equal signs on each diagonal) give two segments, each
 *      cutting off one negative corner, so negative corners never connect
 *      across a face;
 *   3. each segment is directed so that, with m the outward face normal and
 *      w = m x (p2 - p1), w points to the positive side of the face;
 *   4. the directed segments close into loops; each loop is fanned from the
 *      smallest edge index whose fan has no triangle lying inside a single
 *      cube face (a loop through both segments of an ambiguous face could
 *      otherwise give a flat triangle in that face, matched by a mirrored one
 *      in the neighbouring cell).
 * The rule depends only on the four signs of a face, so two cells sharing a
 * face agree on it and meshes are closed.  Step 3 makes every triangle's
 * normal point towards f > 0.
 */
#define OR_MAXT 16
static int or_tab_n[256];
static int or_tab[256][OR_MAXT][3];
static int e_lo[12], e_hi[12], e_axis[12];
static int tab_ready = 0;

static void corner_xyz(int b, int *x) { x[0] = b & 1; x[1] = (b >> 1) & 1; x[2] = (b >> 2) & 1; }

static void build_table(void) {
    for (int e = 0; e < 12; ++e) {
        int ax = e / 4, u = e & 1, v = (e >> 1) & 1, o1 = ax == 0 ? 1 : 0, o2 = ax == 2 ? 1 : 2;
        int c[3] = {0, 0, 0};
        c[o1] = u;
        c[o2] = v;
        e_axis[e] = ax;
        e_lo[e] = c[0] + 2 * c[1] + 4 * c[2];
        e_hi[e] = e_lo[e] + (1 << ax);
    }
    for (int cs = 0; cs < 256; ++cs) {
        int next[12];
        for (int e = 0; e < 12; ++e) next[e] = -1;
        for (int ax = 0; ax < 3; ++ax)
            for (int sd = 0; sd < 2; ++sd) {
                int fe[4], nfe = 0, fc[4], nfc = 0;
                for (int e = 0; e < 12; ++e)
                    if (e_axis[e] != ax && ((e_lo[e] >> ax) & 1) == sd) {
                        int nl = (cs >> e_lo[e]) & 1, nh = (cs >> e_hi[e]) & 1;
                        if (nl != nh) fe[nfe++] = e;
                    }
                for (int b = 0; b < 8; ++b)
                    if (((b >> ax) & 1) == sd) fc[nfc++] = b;
                int segs[2][2], nseg = 0;
                if (nfe == 2) {
                    segs[0][0] = fe[0];
                    segs[0][1] = fe[1];
                    nseg = 1;
                } else if (nfe == 4) {
                    for (int q = 0; q < 4; ++q) {
                        int b = fc[q];
                        if (!((cs >> b) & 1)) continue;
                        int adj[2], na = 0;
                        for (int t = 0; t < 4; ++t)
                            if (e_lo[fe[t]] == b || e_hi[fe[t]] == b) adj[na++] = fe[t];
                        segs[nseg][0] = adj[0];
                        segs[nseg][1] = adj[1];
                        ++nseg;
                    }
                }
                double m[3] = {0, 0, 0};
                m[ax] = sd ? 1.0 : -1.0;
                for (int s = 0; s < nseg; ++s) {
                    int e1 = segs[s][0], e2 = segs[s][1];
                    double p1[3], p2[3];
                    int a1[3], a2[3];
                    corner_xyz(e_lo[e1], a1);
                    corner_xyz(e_lo[e2], a2);
                    for (int a = 0; a < 3; ++a) {
                        p1[a] = 2.0 * a1[a] + (a == e_axis[e1] ? 1.0 : 0.0);
                        p2[a] = 2.0 * a2[a] + (a == e_axis[e2] ? 1.0 : 0.0);
                    }
                    double d[3] = {p2[0] - p1[0], p2[1] - p1[1], p2[2] - p1[2]};
                    double w[3] = {m[1] * d[2] - m[2] * d[1], m[2] * d[0] - m[0] * d[2],
                                   m[0] * d[1] - m[1] * d[0]};
                    /* sides of the segment: +1 and -1; record the signs there */
                    int seen_pos[2] = {0, 0}, seen_neg[2] = {0, 0};
                    for (int q = 0; q < 4; ++q) {
                        int x[3];
                        corner_xyz(fc[q], x);
                        double t = 0;
                        for (int a = 0; a < 3; ++a) t += (2.0 * x[a] - p1[a]) * w[a];
                        int side = t > 0 ? 0 : 1, neg = (cs >> fc[q]) & 1;
                        if (neg) seen_neg[side] = 1; else seen_pos[side] = 1;
                    }
                    int ok;
                    if (seen_pos[0] + seen_neg[0] == 1) ok = seen_pos[0]; /* w side pure */
                    else ok = seen_neg[1];                                /* other side pure */
                    if (ok) next[e1] = e2; else next[e2] = e1;
                }
            }
        int used[12] = {0}, nt = 0;
        for (int e = 0; e < 12; ++e) {
            if (next[e] < 0 || used[e]) continue;
            int loop[12], n = 0, x = e;
            while (!used[x]) {
                used[x] = 1;
                loop[n++] = x;
                x = next[x];
            }
            /* apex: the smallest-index edge of the loop whose fan puts no
             * triangle inside a single cube face (such a triangle would be
             * matched by a mirrored one in the neighbouring cell) */
            int apex = -1;
            for (int cand = 0; cand < 12 && apex < 0; ++cand) {
                int at = -1;
                for (int i = 0; i < n; ++i)
                    if (loop[i] == cand) at = i;
                if (at < 0) continue;
                int flat = 0;
                for (int i = 1; i + 1 < n && !flat; ++i) {
                    int tri[3] = {loop[at], loop[(at + i) % n], loop[(at + i + 1) % n]};
                    for (int ax = 0; ax < 3 && !flat; ++ax)
                        for (int sd = 0; sd < 2 && !flat; ++sd) {
                            int on = 0;
                            for (int v = 0; v < 3; ++v)
                                on += e_axis[tri[v]] != ax && ((e_lo[tri[v]] >> ax) & 1) == sd;
                            flat = on == 3;
                        }
                }
                if (!flat) apex = at;
            }
            if (apex < 0) apex = 0;
            for (int i = 1; i + 1 < n; ++i) {
                or_tab[cs][nt][0] = loop[apex];
                or_tab[cs][nt][1] = loop[(apex + i) % n];
                or_tab[cs][nt][2] = loop[(apex + i + 1) % n];
                ++nt;
            }
        }
        or_tab_n[cs] = nt;
    }
    tab_ready = 1;
}

static void ensure_table(void) {
    if (!tab_ready) {
#pragma omp critical(or_table)
        if (!tab_ready) build_table();
    }
}

/* Copies the table out: ntri[256], edges[256*maxt*3] (-1 padded). */
int or_mc_table(int32_t *ntri, int32_t *edges, int maxt) {
    ensure_table();
    int mx = 0;
    for (int c = 0; c < 256; ++c) {
        ntri[c] = or_tab_n[c];
        if (or_tab_n[c] > mx) mx = or_tab_n[c];
        for (int t = 0; t < maxt; ++t)
            for (int v = 0; v < 3; ++v)
                edges[((size_t)c * maxt + t) * 3 + v] = t < or_tab_n[c] ? or_tab[c][t][v] : -1;
    }
    return mx;
}

/* ------------------------------------------------------------------------ */
/* Growable result buffers                                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t n, cap;
    size_t esz;
    char *p;
} ovec;

static void ov_push(ovec *v, const void *x) {
    if (v->n == v->cap) {
        v->cap = v->cap ? 2 * v->cap : 1024;
        v->p = (char *)realloc(v->p, v->cap * v->esz);
    }
    memcpy(v->p + v->n * v->esz, x, v->esz);
    v->n++;
}

static void ov_cat(ovec *d, const ovec *s) {
    if (!s->n) return;
    if (d->n + s->n > d->cap) {
        d->cap = d->n + s->n;
        d->p = (char *)realloc(d->p, d->cap * d->esz);
    }
    memcpy(d->p + d->n * d->esz, s->p, s->n * s->esz);
    d->n += s->n;
}

/* slots of a result */
enum { R_CELL = 0, R_CASE, R_TKEY, R_TPOS, R_TCELL, R_COLEVAL, R_MARK, R_NSLOT };
static const size_t R_ESZ[R_NSLOT] = {8, 4, 24, 72, 8, 8, 8};

typedef struct {
    ovec v[R_NSLOT];
    double minabs; /* smallest |f| seen at any evaluated corner */
} ores;

static ores *ores_new(void) {
    ores *r = (ores *)calloc(1, sizeof(ores));
    for (int s = 0; s < R_NSLOT; ++s) r->v[s].esz = R_ESZ[s];
    r->minabs = INFINITY;
    return r;
}

int64_t or_res_count(void *h, int slot) { return ((ores *)h)->v[slot].n; }
void or_res_copy(void *h, int slot, void *dst) {
    ores *r = (ores *)h;
    if (r->v[slot].n) memcpy(dst, r->v[slot].p, r->v[slot].n * r->v[slot].esz);
}
double or_res_minabs(void *h) { return ((ores *)h)->minabs; }
void or_res_free(void *h) {
    ores *r = (ores *)h;
    if (!r) return;
    for (int s = 0; s < R_NSLOT; ++s) free(r->v[s].p);
    free(r);
}

static void ores_merge(ores *d, ores *s) {
    for (int k = 0; k < R_NSLOT; ++k) ov_cat(&d->v[k], &s->v[k]);
    if (s->minabs < d->minabs) d->minabs = s->minabs;
}

/* ------------------------------------------------------------------------ */
/* Marching Cubes on one cell                                                */
/* ------------------------------------------------------------------------ */

typedef struct {
    int N;
    double lo[3], h;
} ogrid;

/* Evaluates the 8 corners of cell (i,j,k), returns the case index and, when
 * 0 < case < 255, appends its triangles to r. */
static int mc_cell(const osdb *s, const ogrid *g, int64_t i, int64_t j, int64_t k, ores *r) {
    double fv[8];
    int cs = 0;
    for (int b = 0; b < 8; ++b) {
        int x[3];
        corner_xyz(b, x);
        double p[3] = {g->lo[0] + (double)(i + x[0]) * g->h, g->lo[1] + (double)(j + x[1]) * g->h,
                       g->lo[2] + (double)(k + x[2]) * g->h};
        fv[b] = sdb_eval(s, p);
        if (fabs(fv[b]) < r->minabs) r->minabs = fabs(fv[b]);
        if (fv[b] < 0) cs |= 1 << b;
    }
    if (cs == 0 || cs == 255) return cs;
    int64_t N1 = g->N + 1, cell = (i * g->N + j) * g->N + k;
    for (int t = 0; t < or_tab_n[cs]; ++t) {
        int64_t key[3];
        double pos[9];
        for (int v = 0; v < 3; ++v) {
            int e = or_tab[cs][t][v], x[3];
            corner_xyz(e_lo[e], x);
            int64_t a = i + x[0], b = j + x[1], c = k + x[2];
            key[v] = (int64_t)e_axis[e] * N1 * N1 * N1 + a + N1 * (b + N1 * c);
            double fa = fv[e_lo[e]], fb = fv[e_hi[e]];
            double tt = fa / (fa - fb);
            double pa[3] = {g->lo[0] + (double)a * g->h, g->lo[1] + (double)b * g->h,
                            g->lo[2] + (double)c * g->h};
            pa[e_axis[e]] += tt * g->h;
            pos[3 * v] = pa[0];
            pos[3 * v + 1] = pa[1];
            pos[3 * v + 2] = pa[2];
        }
        ov_push(&r->v[R_TKEY], key);
        ov_push(&r->v[R_TPOS], pos);
        ov_push(&r->v[R_TCELL], &cell);
    }
    return cs;
}

static int grid_of(ogrid *g, int N, const double *lo, double h) {
    if (N < 1 || !(h > 0)) return -1;
    g->N = N;
    g->lo[0] = lo[0];
    g->lo[1] = lo[1];
    g->lo[2] = lo[2];
    g->h = h;
    return 0;
}

/* Marching Cubes on an explicit list of cell ids (i*N + j)*N + k.  Every
 * listed cell gets a case; R_CELL/R_CASE hold all of them in list order. */
void *or_mc(const void *hs, int N, const double *lo, double h, int64_t ncells, const int64_t *cells) {
    const osdb *s = (const osdb *)hs;
    ogrid g;
    if (grid_of(&g, N, lo, h)) return NULL;
    ensure_table();
    ores *out = ores_new();
    int nth = 1;
#ifdef _OPENMP
    nth = omp_get_max_threads();
#endif
    ores **part = (ores **)calloc(nth, sizeof(ores *));
#pragma omp parallel num_threads(nth)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        ores *r = ores_new();
        part[t] = r;
        int64_t lo_i = ncells * t / nth, hi_i = ncells * (t + 1) / nth;
        for (int64_t q = lo_i; q < hi_i; ++q) {
            int64_t c = cells[q], k = c % N, j = (c / N) % N, i = c / ((int64_t)N * N);
            int32_t cs = mc_cell(s, &g, i, j, k, r);
            ov_push(&r->v[R_CELL], &c);
            ov_push(&r->v[R_CASE], &cs);
        }
    }
    for (int t = 0; t < nth; ++t) {
        ores_merge(out, part[t]);
        or_res_free(part[t]);
    }
    free(part);
    return out;
}

/* Enumeration (Sec. 2): Marching Cubes on every cell with kmin <= k < kmax.
 * R_CELL/R_CASE hold the sign-change cells (0 < case < 255) only. */
void *or_enum(const void *hs, int N, const double *lo, double h, int kmin, int kmax) {
    const osdb *s = (const osdb *)hs;
    ogrid g;
    if (grid_of(&g, N, lo, h)) return NULL;
    ensure_table();
    if (kmin < 0) kmin = 0;
    if (kmax > N) kmax = N;
    ores *out = ores_new();
    ores **part = (ores **)calloc(N, sizeof(ores *));
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < N; ++i) {
        ores *r = ores_new();
        for (int j = 0; j < N; ++j)
            for (int k = kmin; k < kmax; ++k) {
                int32_t cs = mc_cell(s, &g, i, j, k, r);
                if (cs != 0 && cs != 255) {
                    int64_t c = ((int64_t)i * N + j) * N + k;
                    ov_push(&r->v[R_CELL], &c);
                    ov_push(&r->v[R_CASE], &cs);
                }
            }
        part[i] = r;
    }
    for (int i = 0; i < N; ++i) {
        ores_merge(out, part[i]);
        or_res_free(part[i]);
    }
    free(part);
    return out;
}

/* ------------------------------------------------------------------------ */
/* Grid hopping (Sec. 3, Algorithm 1)                                        */
/* ------------------------------------------------------------------------ */
/*
 * One ray per column (i,j) through the cell centres (Eq. 1-2), cast along
 * +z from k = 0.  At cell k the bound d = |f(centre_k)| is taken (Eq. 3); a
 * cell with d <= tau gets polygonized and the ray moves on by one cell
 * (Algorithm 1 polygonizes the cell it lands in, then increments k);
 * otherwise the ray jumps floor(d / h) cells at once, at least one, because
 * sphere tracing by d can not pass the surface and the discrete jump is the
 * part of that step that lands on a cell centre.  tau is the polygonization
 * distance of Eq. 4 expressed in cells of size h: the default is one cell
 * diagonal, sqrt(3) h; tau_mode 1 uses half a diagonal.  eps > 0 shrinks
 * every bound first, d = max(|f| - eps, 0), as a reduced-precision evaluator
 * must.
 * Result: R_MARK = marked cell ids in column order, R_COLEVAL = evaluations
 * per listed column.
 */
void *or_hop(const void *hs, int N, const double *lo, double h, double tau, double eps, int64_t ncols,
             const int64_t *cols) {
    const osdb *s = (const osdb *)hs;
    ogrid g;
    if (grid_of(&g, N, lo, h)) return NULL;
    int64_t nc = cols ? ncols : (int64_t)N * N;
    ores *out = ores_new();
    int64_t *ev = (int64_t *)calloc(nc ? nc : 1, sizeof(int64_t));
    int nth = 1;
#ifdef _OPENMP
    nth = omp_get_max_threads();
#endif
    ores **part = (ores **)calloc(nth, sizeof(ores *));
#pragma omp parallel num_threads(nth)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        ores *r = ores_new();
        part[t] = r;
        int64_t c0 = nc * t / nth, c1 = nc * (t + 1) / nth;
        for (int64_t q = c0; q < c1; ++q) {
            int64_t col = cols ? cols[q] : q, i = col / N, j = col % N;
            double x = g.lo[0] + ((double)i + 0.5) * g.h, y = g.lo[1] + ((double)j + 0.5) * g.h;
            int64_t k = 0, n = 0;
            while (k < N) {
                double p[3] = {x, y, g.lo[2] + ((double)k + 0.5) * g.h};
                double d = fabs(sdb_eval(s, p));
                ++n;
                if (eps > 0) d = d > eps ? d - eps : 0.0;
                if (d <= tau) {
                    int64_t cell = col * N + k;
                    ov_push(&r->v[R_MARK], &cell);
                    k += 1;
                } else {
                    double st = floor(d / g.h);
                    k += st < 1.0 ? 1 : (st > (double)N ? (int64_t)N : (int64_t)st);
                }
            }
            ev[q] = n;
        }
    }
    for (int t = 0; t < nth; ++t) {
        ores_merge(out, part[t]);
        or_res_free(part[t]);
    }
    free(part);
    for (int64_t q = 0; q < nc; ++q) ov_push(&out->v[R_COLEVAL], &ev[q]);
    free(ev);
    return out;
}

/* ------------------------------------------------------------------------ */
/* Gradients of the neural SDB (implicit-surface adjoint)                   */
/* ------------------------------------------------------------------------ */
/*
 * For f(p; theta) = (rad |p| - r0 + alpha g(p; theta)) / (beta lam):
 *   grad_x f = (rad p/|p| + alpha dg/dp) / (beta lam)
 *   df/dtheta = alpha dg/dtheta / (beta lam)
 * by back-propagation through the ReLU layers.  A vertex v on the level set
 * f = 0 moves with theta as dv/dtheta = -grad_x f (df/dtheta) / |grad_x f|^2,
 * so for a loss L(v):
 *   dL/dtheta = sum_v s_v df/dtheta(v),  s_v = -(dL/dv . grad_x f)/|grad_x f|^2.
 * Parameters are packed like the MLP parameter block of or_mlp_new.
 */
static void mlp_grads(const osdb *s, const double *p, double *gx, double *gth, double scale) {
    int W = s->width, L = s->nmid;
    double *z = (double *)malloc(sizeof(double) * (size_t)(L + 1) * W);
    double *dl = (double *)malloc(sizeof(double) * 2 * W), *dn = dl + W;
    (void)mlp_g(s, p, z);
    double c = s->alpha / (s->beta * s->lam);
    /* offsets inside the packed parameter vector */
    size_t oW0 = 0, ob0 = (size_t)3 * W, omid = ob0 + W, ow = omid + (size_t)L * ((size_t)W * W + W);
    /* output layer: g = wout . a_L + bout */
    const double *aL = z + (size_t)L * W;
    for (int i = 0; i < W; ++i) {
        double a = aL[i] > 0 ? aL[i] : 0.0;
        if (gth) gth[ow + i] += scale * c * a;
        dl[i] = aL[i] > 0 ? s->wout[i] : 0.0; /* dg/dz_L */
    }
    if (gth) gth[ow + W] += scale * c;
    for (int l = L - 1; l >= 0; --l) {
        const double *Wl = s->Wm[l];
        const double *zin = z + (size_t)l * W;
        size_t oWl = omid + (size_t)l * ((size_t)W * W + W), obl = oWl + (size_t)W * W;
        for (int o = 0; o < W; ++o) {
            if (gth) {
                gth[obl + o] += scale * c * dl[o];
                for (int i = 0; i < W; ++i) {
                    double a = zin[i] > 0 ? zin[i] : 0.0;
                    gth[oWl + (size_t)o * W + i] += scale * c * dl[o] * a;
                }
            }
        }
        for (int i = 0; i < W; ++i) {
            double acc = 0;
            for (int o = 0; o < W; ++o) acc += Wl[(size_t)o * W + i] * dl[o];
            dn[i] = zin[i] > 0 ? acc : 0.0;
        }
        memcpy(dl, dn, sizeof(double) * W);
    }
    double dgp[3] = {0, 0, 0};
    for (int o = 0; o < W; ++o) {
        if (gth) {
            gth[ob0 + o] += scale * c * dl[o];
            for (int a = 0; a < 3; ++a) gth[oW0 + 3 * (size_t)o + a] += scale * c * dl[o] * p[a];
        }
        for (int a = 0; a < 3; ++a) dgp[a] += s->W0[3 * o + a] * dl[o];
    }
    double r = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    for (int a = 0; a < 3; ++a)
        gx[a] = (s->rad * (r > 0 ? p[a] / r : 0.0) + s->alpha * dgp[a]) / (s->beta * s->lam);
    free(z);
    free(dl);
}

/* grad_x f at n points: gx[n,3] */
int or_grad_x(const void *hs, int64_t n, const double *p, double *gx) {
    const osdb *s = (const osdb *)hs;
    if (s->kind != 1) return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) mlp_grads(s, p + 3 * i, gx + 3 * i, NULL, 0.0);
    return 0;
}

/* df/dtheta at one point, packed like the parameter block. */
int or_grad_theta_point(const void *hs, const double *p, double *gth, int64_t nparam) {
    const osdb *s = (const osdb *)hs;
    if (s->kind != 1) return -1;
    double gx[3];
    memset(gth, 0, sizeof(double) * nparam);
    mlp_grads(s, p, gx, gth, 1.0);
    return 0;
}

/* Implicit adjoint: dL/dtheta = sum_v s_v df/dtheta(v). */
int or_adjoint(const void *hs, int64_t nv, const double *v, const double *dldv, double *gth, int64_t nparam) {
    const osdb *s = (const osdb *)hs;
    if (s->kind != 1) return -1;
    int nth = 1;
#ifdef _OPENMP
    nth = omp_get_max_threads();
#endif
    double *acc = (double *)calloc((size_t)nth * nparam, sizeof(double));
#pragma omp parallel num_threads(nth)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        double *mine = acc + (size_t)t * nparam;
        int64_t a0 = nv * t / nth, a1 = nv * (t + 1) / nth;
        for (int64_t q = a0; q < a1; ++q) {
            double gx[3];
            mlp_grads(s, v + 3 * q, gx, NULL, 0.0);
            double g2 = gx[0] * gx[0] + gx[1] * gx[1] + gx[2] * gx[2];
            double sv = -(dldv[3 * q] * gx[0] + dldv[3 * q + 1] * gx[1] + dldv[3 * q + 2] * gx[2]) / g2;
            mlp_grads(s, v + 3 * q, gx, mine, sv);
        }
    }
    memset(gth, 0, sizeof(double) * nparam);
    for (int t = 0; t < nth; ++t)
        for (int64_t i = 0; i < nparam; ++i) gth[i] += acc[(size_t)t * nparam + i];
    free(acc);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of an analytic (CSG) SDB                                          */
/* ------------------------------------------------------------------------ */
/*
 * A min / max fold selects one primitive at each point (union keeps the
 * running value unless the new distance is strictly smaller, subtraction and
 * intersection unless it is strictly larger), so f = sgn * d_a(p) with
 * sgn = -1 when the selected primitive was subtracted.  Gradients of the
 * exact distances with respect to the point, the centre c (the negative of the
 * point gradient) and the size parameters:
 *   sphere  d = |p - c| - r:                 dd/dr = -1
 *   torus   a = |(qx,qz)| - R, d = |(a,qy)| - r:  dd/dR = -a/|(a,qy)|, dd/dr = -1
 *   box     e = |q| - h; outside: d = |max(e,0)|, dd/dh = -max(e,0)/d;
 *           inside: d = max_k e_k, dd/dh_k = -1 for the largest k
 * with q = Rot (p - c) and dd/dp = Rot^T dd/dq.
 * Output per primitive (17 doubles like the primitive rows): dL/dc in slots
 * 2..4, dL/dparam in slots 5..7, everything else 0.
 */
static double prim_grad(const double *pr, const double *p, double *gp /*dd/dp*/, double *gs /*dd/dparam*/) {
    const double *c = pr + 2, *prm = pr + 5, *R = pr + 8;
    double d[3] = {p[0] - c[0], p[1] - c[1], p[2] - c[2]}, q[3], gq[3] = {0, 0, 0}, val;
    for (int r = 0; r < 3; ++r) q[r] = R[3 * r] * d[0] + R[3 * r + 1] * d[1] + R[3 * r + 2] * d[2];
    gs[0] = gs[1] = gs[2] = 0.0;
    switch ((int)pr[0]) {
    case OR_SPHERE: {
        double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
        val = n - prm[0];
        for (int a = 0; a < 3; ++a) gq[a] = n > 0 ? q[a] / n : 0.0;
        gs[0] = -1.0;
        break;
    }
    case OR_TORUS: {
        double rxz = sqrt(q[0] * q[0] + q[2] * q[2]);
        double a = rxz - prm[0];
        double n = sqrt(a * a + q[1] * q[1]);
        val = n - prm[1];
        if (n > 0) {
            gq[0] = rxz > 0 ? a * q[0] / (rxz * n) : 0.0;
            gq[1] = q[1] / n;
            gq[2] = rxz > 0 ? a * q[2] / (rxz * n) : 0.0;
            gs[0] = -a / n;
        }
        gs[1] = -1.0;
        break;
    }
    case OR_CAPSULE:
    case OR_CYLINDER:
    case OR_HEXPRISM:
    case OR_CONE: {
        /* derivatives of these piecewise-smooth distances by central
         * differences of the closed forms above (step 1e-7 of the unit
         * domain; FP64 keeps them to about 1e-9) */
        double pp[17], hh = 1e-7;
        for (int i = 0; i < 17; ++i) pp[i] = pr[i];
        val = prim_eval(pr, p);
        for (int a = 0; a < 3; ++a) {
            double hi_[3] = {p[0], p[1], p[2]}, lo_[3] = {p[0], p[1], p[2]};
            hi_[a] += hh;
            lo_[a] -= hh;
            gq[a] = 0.0;
            gs[a] = 0.0;
            double dh = prim_eval(pr, hi_), dl = prim_eval(pr, lo_);
            gp[a] = (dh - dl) / (2 * hh);
        }
        for (int a = 0; a < 2; ++a) {
            pp[5 + a] = pr[5 + a] + hh;
            double dh = prim_eval(pp, p);
            pp[5 + a] = pr[5 + a] - hh;
            double dl = prim_eval(pp, p);
            pp[5 + a] = pr[5 + a];
            gs[a] = (dh - dl) / (2 * hh);
        }
        return val;
    }
    default: {
        double e[3], o2 = 0.0;
        int km = 0;
        for (int a = 0; a < 3; ++a) {
            e[a] = fabs(q[a]) - prm[a];
            if (e[a] > 0) o2 += e[a] * e[a];
            if (e[a] > e[km]) km = a;
        }
        if (o2 > 0) {
            double n = sqrt(o2);
            val = n;
            for (int a = 0; a < 3; ++a) {
                double m = e[a] > 0 ? e[a] / n : 0.0;
                gq[a] = (q[a] < 0 ? -1.0 : 1.0) * m;
                gs[a] = -m;
            }
        } else {
            val = e[km];
            gq[km] = q[km] < 0 ? -1.0 : 1.0;
            gs[km] = -1.0;
        }
        break;
    }
    }
    for (int a = 0; a < 3; ++a) gp[a] = R[a] * gq[0] + R[3 + a] * gq[1] + R[6 + a] * gq[2];
    return val;
}

int or_csg_adjoint(const void *hs, int64_t nv, const double *v, const double *dldv, double *out) {
    const osdb *s = (const osdb *)hs;
    if (s->kind != 0) return -1;
    int nth = 1;
#ifdef _OPENMP
    nth = omp_get_max_threads();
#endif
    size_t np = (size_t)s->nprim * OR_PRIM_STRIDE;
    double *acc = (double *)calloc((size_t)nth * np, sizeof(double));
#pragma omp parallel num_threads(nth)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        double *mine = acc + (size_t)t * np;
        int64_t a0 = nv * t / nth, a1 = nv * (t + 1) / nth;
        for (int64_t qv = a0; qv < a1; ++qv) {
            const double *p = v + 3 * qv;
            int act = 0;
            double sgn = 1.0, f = prim_eval(s->prim, p);
            for (int n = 1; n < s->nprim; ++n) {
                const double *pr = s->prim + (size_t)n * OR_PRIM_STRIDE;
                double d = prim_eval(pr, p);
                int op = (int)pr[1];
                if (op == OR_UNION) {
                    if (d < f) { f = d; act = n; sgn = 1.0; }
                } else if (op == OR_SUBTRACT) {
                    if (-d > f) { f = -d; act = n; sgn = -1.0; }
                } else {
                    if (d > f) { f = d; act = n; sgn = 1.0; }
                }
            }
            double gp[3], gs[3];
            prim_grad(s->prim + (size_t)act * OR_PRIM_STRIDE, p, gp, gs);
            double gx[3] = {sgn * gp[0], sgn * gp[1], sgn * gp[2]};
            double g2 = gx[0] * gx[0] + gx[1] * gx[1] + gx[2] * gx[2];
            if (!(g2 > 0)) continue;
            double sv = -(dldv[3 * qv] * gx[0] + dldv[3 * qv + 1] * gx[1] + dldv[3 * qv + 2] * gx[2]) / g2;
            double *o = mine + (size_t)act * OR_PRIM_STRIDE;
            for (int a = 0; a < 3; ++a) {
                o[2 + a] += sv * (-gx[a]);     /* df/dc = -sgn dd/dp */
                o[5 + a] += sv * sgn * gs[a];
            }
        }
    }
    memset(out, 0, sizeof(double) * np);
    for (int t = 0; t < nth; ++t)
        for (size_t i = 0; i < np; ++i) out[i] += acc[(size_t)t * np + i];
    free(acc);
    return 0;
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Sets the number of host threads later oracle calls use (n < 1: all cores).
 * Harness control only (timing a one-core run); no arithmetic changes. */
void or_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n >= 1 ? n : omp_get_num_procs());
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Continuation (Sec. 2): crawl the surface from seed cells                   */
/* ------------------------------------------------------------------------ */
/*
 * The comparison method of Sec. 2 and 5.1: starting from a seed cell that
 * the surface passes through, cells are propagated across the surface until
 * the surface is closed; each seed gives (at most) one mesh component.  A
 * cell's surface leaves it through exactly the faces whose four corners do
 * not all have one sign, so the neighbour across each such face is a surface
 * cell too and joins the queue (breadth first, each cell once).
 * Seeds are points: from the cell (i0, j0, k0) holding the point, the lattice
 * vertices (a, j0, k0), a = i0 .. N, are scanned in +x order and the first
 * pair with a sign change gives the seed cell (a, j0, k0) (Bloomenthal's
 * search for a seed from a point); a point whose line has no sign change
 * gives none.
 * Result: R_CELL / R_CASE the visited cells in visit order, the triangles of
 * each (Marching Cubes as in or_mc), R_COLEVAL one entry per seed: the seed
 * cell id or -1.
 */
static double corner_val(const osdb *s, const ogrid *g, int64_t a, int64_t b, int64_t c) {
    double p[3] = {g->lo[0] + (double)a * g->h, g->lo[1] + (double)b * g->h, g->lo[2] + (double)c * g->h};
    return sdb_eval(s, p);
}

void *or_cont(const void *hs, int N, const double *lo, double h, int64_t nseeds, const double *seeds) {
    const osdb *s = (const osdb *)hs;
    ogrid g;
    if (grid_of(&g, N, lo, h)) return NULL;
    ensure_table();
    ores *out = ores_new();
    const int64_t NN = N, ncell = NN * NN * NN;
    uint64_t *vis = (uint64_t *)calloc((size_t)(ncell / 64 + 1), sizeof(uint64_t));
    ovec q = {0, 0, 8, NULL};
    for (int64_t sd = 0; sd < nseeds; ++sd) {
        int64_t ijk[3], found = -1;
        for (int a = 0; a < 3; ++a) {
            double x = floor((seeds[3 * sd + a] - g.lo[a]) / g.h);
            ijk[a] = x < 0 ? 0 : (x > NN - 1 ? NN - 1 : (int64_t)x);
        }
        double fprev = corner_val(s, &g, ijk[0], ijk[1], ijk[2]);
        for (int64_t a = ijk[0]; a < NN; ++a) {
            double fnext = corner_val(s, &g, a + 1, ijk[1], ijk[2]);
            if ((fprev < 0) != (fnext < 0)) {
                found = (a * NN + ijk[1]) * NN + ijk[2];
                break;
            }
            fprev = fnext;
        }
        ov_push(&out->v[R_COLEVAL], &found);
        if (found >= 0 && !(vis[found >> 6] >> (found & 63) & 1)) {
            vis[found >> 6] |= 1ull << (found & 63);
            ov_push(&q, &found);
        }
    }
    for (int64_t head = 0; head < q.n; ++head) {
        int64_t c = ((int64_t *)q.p)[head];
        int64_t k = c % NN, j = (c / NN) % NN, i = c / (NN * NN);
        double fv[8];
        for (int b = 0; b < 8; ++b) {
            int x[3];
            corner_xyz(b, x);
            fv[b] = corner_val(s, &g, i + x[0], j + x[1], k + x[2]);
        }
        int32_t cs = mc_cell(s, &g, i, j, k, out);
        ov_push(&out->v[R_CELL], &c);
        ov_push(&out->v[R_CASE], &cs);
        for (int ax = 0; ax < 3; ++ax)
            for (int side = 0; side < 2; ++side) {
                int neg = 0;
                for (int b = 0; b < 8; ++b)
                    if (((b >> ax) & 1) == side) neg += fv[b] < 0;
                if (neg == 0 || neg == 4) continue; /* the surface does not cross this face */
                int64_t n3[3] = {i, j, k};
                n3[ax] += side ? 1 : -1;
                if (n3[ax] < 0 || n3[ax] >= NN) continue;
                int64_t nc = (n3[0] * NN + n3[1]) * NN + n3[2];
                if (vis[nc >> 6] >> (nc & 63) & 1) continue;
                vis[nc >> 6] |= 1ull << (nc & 63);
                ov_push(&q, &nc);
            }
    }
    free(q.p);
    free(vis);
    return out;
}
