/*
 * FP64 CPU oracle of one differentiable 3D Gaussian Splatting mapping iteration
 * (CaRtGS, arXiv 2410.00486).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may call, link or load
 * this file: only the tests, the smoke check and the benchmark's CPU-baseline leg
 * use it.  It shares no code, header or constant table with the CUDA path.
 *
 * It is a plain, slow restatement of the definitions, evaluated in double
 * precision, one Gaussian / one pixel at a time:
 *   - preprocess  : 3DGS projection of a Gaussian to the image plane, the
 *                   "projected 2D Gaussian" of Eq. 1 (Sec. III-B), plus the
 *                   SH colour c_k of Eq. 1.
 *   - bin         : per-tile lists ordered by depth ("each thread in a tile",
 *                   Sec. III-C.1; splats blended in depth order, Eq. 1).
 *   - render_fwd  : alpha blending, Eq. 1 (Sec. III-B), read with (1 - alpha_j)
 *                   inside the product; plus the L1 photometric/depth loss (the
 *                   L1 part of Eq. 9).
 *   - render_bwd  : Eqs. 2-4 (Sec. III-C.1): per (splat, pixel) gradient terms,
 *                   summed over the pixels a splat touches.  Transmittances are
 *                   kept from a forward re-walk of each pixel (no division) and
 *                   the "colour behind" is an explicit suffix sum.
 *   - preprocess_bwd : chain rule from the projected quantities back to
 *                   position, scale, rotation, opacity and SH (Sec. III-B lists
 *                   the parameters), summed over the views of the window.
 *   - densify_stats  : per-Gaussian view-space positional-gradient statistics
 *                   that guide densification (Sec. III-A.3, Sec. IV-A).
 * Adam and the keyframe scheduler live in oracle.py.
 *
 * Threads (OpenMP, orc_set_threads): loops run in parallel only over outputs that no
 * other iteration writes (views, Gaussians, rows, listed pixels), and sums that cross
 * iterations are formed per row and added in a fixed order, so every result is the same
 * bit for bit whatever the thread count; the arithmetic of each step is unchanged.
 *
 * Readings where the paper is silent (it defers to 3DGS for the renderer) are
 * listed beside each step.  Layouts:
 *   params  : means[n][3] | log_scales[n][3] | quats[n][4] (w,x,y,z) |
 *             opacity_logits[n] | sh_dc[n][3] | sh_rest[n][K-1][3]
 *   cams    : double[V][17] = R[9] (world->camera, row-major), t[3],
 *             fx, fy, cx, cy, loss weight
 *   records : double[V*n][10] = u, v, conicA, conicB, conicC, opacity, r, g, b, depth
 *   slot grads : double[V*n][10], derivatives w.r.t. the record fields
 *   a "slot" is (view v, Gaussian g) -> index v*n + g
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NREC 10
#define NCAM 17

/* ------------------------------------------------------------------ helpers */

/* Number of OpenMP threads the loops below use (default: OpenMP's own, all cores). */
void orc_set_threads(int k) { if (k > 0) omp_set_num_threads(k); }
int orc_get_threads(void) { return omp_get_max_threads(); }

static int64_t sh_count(int deg) { return (int64_t)(deg + 1) * (deg + 1); }

typedef struct { int64_t means, scales, quats, opac, dc, rest, total; } layout_t;

static layout_t param_layout(int64_t n, int deg)
{
    layout_t L;
    int64_t K = sh_count(deg);
    L.means = 0;
    L.scales = 3 * n;
    L.quats = 6 * n;
    L.opac = 10 * n;
    L.dc = 11 * n;
    L.rest = 14 * n;
    L.total = 14 * n + 3 * (K - 1) * n;
    return L;
}

/* c = a (ra x ca) * b (ca x cb), row-major */
static void matmul(const double *a, const double *b, double *c, int ra, int ca, int cb)
{
    for (int i = 0; i < ra; i++)
        for (int j = 0; j < cb; j++) {
            double s = 0.0;
            for (int k = 0; k < ca; k++) s += a[i * ca + k] * b[k * cb + j];
            c[i * cb + j] = s;
        }
}

static void transpose(const double *a, double *t, int r, int c)
{
    for (int i = 0; i < r; i++)
        for (int j = 0; j < c; j++) t[j * r + i] = a[i * c + j];
}

/* Unit quaternion (w, x, y, z) -> rotation matrix (standard formula). */
static void quat_rot(const double q[4], double R[9])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* dR/dq_k for k = w, x, y, z (each a 3x3 row-major matrix), at a unit q. */
static void quat_rot_jac(const double q[4], double dR[4][9])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double dw[9] = {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0};
    double dx[9] = {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x};
    double dy[9] = {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y};
    double dz[9] = {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0};
    memcpy(dR[0], dw, sizeof dw);
    memcpy(dR[1], dx, sizeof dx);
    memcpy(dR[2], dy, sizeof dy);
    memcpy(dR[3], dz, sizeof dz);
}

/*
 * Real spherical harmonics up to degree 3, Condon-Shortley phase kept, ordered
 * m = -l..l within each band (the convention of 3DGS, which the paper keeps,
 * Sec. III-B: "SH in R^48" = 16 coefficients x RGB).  Constants are written from
 * their closed forms.  Y[k] at a unit direction (x, y, z); dY[k][3] its gradient
 * w.r.t. (x, y, z) treated as free variables.
 */
static void sh_basis(int deg, double x, double y, double z, double Y[16], double dY[16][3])
{
    const double pi = 3.14159265358979323846;
    memset(Y, 0, 16 * sizeof(double));
    memset(dY, 0, 16 * 3 * sizeof(double));
    Y[0] = 0.5 * sqrt(1.0 / pi);
    if (deg < 1) return;
    double c1 = sqrt(3.0 / (4.0 * pi));
    Y[1] = -c1 * y; dY[1][1] = -c1;
    Y[2] = c1 * z;  dY[2][2] = c1;
    Y[3] = -c1 * x; dY[3][0] = -c1;
    if (deg < 2) return;
    double xx = x * x, yy = y * y, zz = z * z;
    double a = 0.5 * sqrt(15.0 / pi), b = 0.25 * sqrt(5.0 / pi), c = 0.25 * sqrt(15.0 / pi);
    Y[4] = a * x * y;               dY[4][0] = a * y;       dY[4][1] = a * x;
    Y[5] = -a * y * z;              dY[5][1] = -a * z;      dY[5][2] = -a * y;
    Y[6] = b * (2 * zz - xx - yy);  dY[6][0] = -2 * b * x;  dY[6][1] = -2 * b * y; dY[6][2] = 4 * b * z;
    Y[7] = -a * x * z;              dY[7][0] = -a * z;      dY[7][2] = -a * x;
    Y[8] = c * (xx - yy);           dY[8][0] = 2 * c * x;   dY[8][1] = -2 * c * y;
    if (deg < 3) return;
    double d0 = 0.25 * sqrt(35.0 / (2 * pi)), d1 = 0.5 * sqrt(105.0 / pi);
    double d2 = 0.25 * sqrt(21.0 / (2 * pi)), d3 = 0.25 * sqrt(7.0 / pi), d5 = 0.25 * sqrt(105.0 / pi);
    Y[9] = -d0 * y * (3 * xx - yy);
    dY[9][0] = -6 * d0 * x * y;     dY[9][1] = -d0 * (3 * xx - 3 * yy);
    Y[10] = d1 * x * y * z;
    dY[10][0] = d1 * y * z;         dY[10][1] = d1 * x * z; dY[10][2] = d1 * x * y;
    Y[11] = -d2 * y * (4 * zz - xx - yy);
    dY[11][0] = 2 * d2 * x * y;     dY[11][1] = -d2 * (4 * zz - xx - 3 * yy); dY[11][2] = -8 * d2 * y * z;
    Y[12] = d3 * z * (2 * zz - 3 * xx - 3 * yy);
    dY[12][0] = -6 * d3 * x * z;    dY[12][1] = -6 * d3 * y * z; dY[12][2] = d3 * (6 * zz - 3 * xx - 3 * yy);
    Y[13] = -d2 * x * (4 * zz - xx - yy);
    dY[13][0] = -d2 * (4 * zz - 3 * xx - yy); dY[13][1] = 2 * d2 * x * y; dY[13][2] = -8 * d2 * x * z;
    Y[14] = d5 * z * (xx - yy);
    dY[14][0] = 2 * d5 * x * z;     dY[14][1] = -2 * d5 * y * z; dY[14][2] = d5 * (xx - yy);
    Y[15] = -d0 * x * (xx - 3 * yy);
    dY[15][0] = -d0 * (3 * xx - 3 * yy); dY[15][1] = 6 * d0 * x * y;
}

/* exported for the basis pin test: Y[16], dY[48] */
void orc_sh_basis(int deg, double x, double y, double z, double *Y, double *dY)
{
    double dd[16][3];
    sh_basis(deg, x, y, z, Y, dd);
    memcpy(dY, dd, sizeof dd);
}

/* ---------------------------------------------------------------- projection */

/* Everything the forward computes for one (view, Gaussian), kept for the backward. */
typedef struct {
    int visible;          /* 0 = culled (behind near plane, det <= 0, empty rect) */
    double s[3], qn[4], qnorm, R[9], M[9], Sigma[9];
    double t[3], J[6], xclamped, yclamped, xsign, ysign, limx, limy;
    double Tm[6], a, b, c, det, conA, conB, conC;
    double lam, r3;       /* largest eigenvalue, 3*sqrt(lam) */
    int radius;
    double u, v;
    double d[3], dnorm, dir[3], Y[16], dY[16][3], rgb[3];
    int clampmask;
    double opacity;
    int rect[4];          /* x_lo, x_hi, y_lo, y_hi (tile indices, hi exclusive) */
} proj_t;

static int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* floor(k / B) for an integer k of either sign */
static int floordiv(long k, int B) { return (int)floor((double)k / (double)B); }

/*
 * Tile rectangle of a splat with centre (u, v) and integer radius r (reading of the
 * 3DGS binning rule: tiles overlapping the square [u-r, u+r] x [v-r, v+r]):
 *   x_lo = clamp(floor((u - r) / B), 0, Tx), x_hi = clamp(floor((u + r + B - 1) / B), 0, Tx)
 * which, since r and B are integers, equals the same expression with u replaced
 * by floor(u).  Likewise in y.
 */
static void tile_rect(double u, double v, int r, int B, int Tx, int Ty, int rect[4])
{
    long fu = (long)floor(u), fv = (long)floor(v);
    rect[0] = clampi(floordiv(fu - r, B), 0, Tx);
    rect[1] = clampi(floordiv(fu + r + B - 1, B), 0, Tx);
    rect[2] = clampi(floordiv(fv - r, B), 0, Ty);
    rect[3] = clampi(floordiv(fv + r + B - 1, B), 0, Ty);
}

static void project(const double *P, int64_t n, int deg, int64_t g, const double *cam,
                    int W, int H, int B, double near_z, proj_t *o)
{
    layout_t L = param_layout(n, deg);
    int64_t K = sh_count(deg);
    memset(o, 0, sizeof *o);
    const double *Rc = cam, *tc = cam + 9;
    double fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15];
    const double *p = P + L.means + 3 * g;

    /* camera-space position t = Rc p + tc; near-plane cull (reading: near = 0.2) */
    for (int i = 0; i < 3; i++) o->t[i] = Rc[3 * i] * p[0] + Rc[3 * i + 1] * p[1] + Rc[3 * i + 2] * p[2] + tc[i];
    if (!(o->t[2] > near_z)) return;

    /* activations: s = exp(log s), unit quaternion, sigmoid opacity */
    for (int i = 0; i < 3; i++) o->s[i] = exp(P[L.scales + 3 * g + i]);
    const double *q = P + L.quats + 4 * g;
    o->qnorm = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; i++) o->qn[i] = q[i] / o->qnorm;
    o->opacity = 1.0 / (1.0 + exp(-P[L.opac + g]));

    /* world covariance Sigma = (R S)(R S)^T */
    quat_rot(o->qn, o->R);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) o->M[3 * i + j] = o->R[3 * i + j] * o->s[j];
    double Mt[9];
    transpose(o->M, Mt, 3, 3);
    matmul(o->M, Mt, o->Sigma, 3, 3, 3);

    /* EWA: Jacobian of the perspective map at t, with the 3DGS guard band (1.3 x half-FoV) */
    double tz = o->t[2];
    o->limx = 1.3 * (0.5 * W / fx);
    o->limy = 1.3 * (0.5 * H / fy);
    double rx = o->t[0] / tz, ry = o->t[1] / tz;
    o->xclamped = (rx > o->limx || rx < -o->limx);
    o->yclamped = (ry > o->limy || ry < -o->limy);
    o->xsign = rx > 0 ? 1.0 : -1.0;
    o->ysign = ry > 0 ? 1.0 : -1.0;
    double xc = (o->xclamped ? o->xsign * o->limx : rx) * tz;
    double yc = (o->yclamped ? o->ysign * o->limy : ry) * tz;
    o->J[0] = fx / tz; o->J[1] = 0.0;     o->J[2] = -fx * xc / (tz * tz);
    o->J[3] = 0.0;     o->J[4] = fy / tz; o->J[5] = -fy * yc / (tz * tz);
    matmul(o->J, Rc, o->Tm, 2, 3, 3);
    double TS[6], Tt[6], cov[4];
    matmul(o->Tm, o->Sigma, TS, 2, 3, 3);
    transpose(o->Tm, Tt, 2, 3);
    matmul(TS, Tt, cov, 2, 3, 2);
    /* low-pass filter: + 0.3 I (reading, 3DGS) */
    o->a = cov[0] + 0.3;
    o->b = cov[1];
    o->c = cov[3] + 0.3;
    o->det = o->a * o->c - o->b * o->b;
    if (!(o->det > 0.0)) return;
    o->conA = o->c / o->det;
    o->conB = -o->b / o->det;
    o->conC = o->a / o->det;

    /* 3-sigma radius of the larger eigenvalue (reading: opacity independent) */
    double mid = 0.5 * (o->a + o->c);
    double disc = mid * mid - o->det;
    o->lam = mid + sqrt(disc > 0.1 ? disc : 0.1);
    o->r3 = 3.0 * sqrt(o->lam);
    o->radius = (int)ceil(o->r3);

    o->u = fx * o->t[0] / tz + cx;
    o->v = fy * o->t[1] / tz + cy;
    int Tx = (W + B - 1) / B, Ty = (H + B - 1) / B;
    tile_rect(o->u, o->v, o->radius, B, Tx, Ty, o->rect);
    if ((o->rect[1] - o->rect[0]) * (o->rect[3] - o->rect[2]) == 0) return;

    /* view-dependent colour: direction from the camera centre to the mean, SH + 0.5,
     * clamped below at 0 (reading: no upper clamp), clamp mask kept for the backward */
    double cpos[3];
    for (int i = 0; i < 3; i++) cpos[i] = -(Rc[i] * tc[0] + Rc[3 + i] * tc[1] + Rc[6 + i] * tc[2]);
    for (int i = 0; i < 3; i++) o->d[i] = p[i] - cpos[i];
    o->dnorm = sqrt(o->d[0] * o->d[0] + o->d[1] * o->d[1] + o->d[2] * o->d[2]);
    for (int i = 0; i < 3; i++) o->dir[i] = o->d[i] / o->dnorm;
    sh_basis(deg, o->dir[0], o->dir[1], o->dir[2], o->Y, o->dY);
    for (int ch = 0; ch < 3; ch++) {
        double acc = o->Y[0] * P[L.dc + 3 * g + ch];
        for (int k = 1; k < K; k++) acc += o->Y[k] * P[L.rest + (3 * (K - 1)) * g + 3 * (k - 1) + ch];
        acc += 0.5;
        if (acc < 0.0) { acc = 0.0; o->clampmask |= 1 << ch; }
        o->rgb[ch] = acc;
    }
    o->visible = 1;
}

/*
 * Per (view, Gaussian) projection.  Outputs per slot: the 10-field record, the radius
 * (0 = culled), the tile rect, the colour clamp mask and a "fragile" flag: set when
 * a rounding-sized change of u, v or 3*sqrt(lambda) would move the tile rect (so a
 * float32 evaluation may legitimately bin the splat differently).  `tol_px` is that
 * rounding size in pixels.
 */
int orc_preprocess(const double *P, int64_t n, int deg, const double *cams, int V,
                   int W, int H, int B, double near_z, double tol_px,
                   double *rec, int32_t *radius, int32_t *rect, int32_t *clampmask,
                   int32_t *fragile)
{
    int Tx = (W + B - 1) / B, Ty = (H + B - 1) / B;
    for (int v = 0; v < V; v++)
#pragma omp parallel for schedule(static)
        for (int64_t g = 0; g < n; g++) {
            proj_t o;
            int64_t s = (int64_t)v * n + g;
            project(P, n, deg, g, cams + NCAM * v, W, H, B, near_z, &o);
            double *r = rec + NREC * s;
            memset(r, 0, NREC * sizeof(double));
            rect[4 * s] = rect[4 * s + 1] = rect[4 * s + 2] = rect[4 * s + 3] = 0;
            radius[s] = 0;
            clampmask[s] = 0;
            fragile[s] = 0;
            /* near-plane decision close to the threshold */
            if (fabs(o.t[2] - near_z) < 1e-6 * (1.0 + fabs(near_z))) fragile[s] = 1;
            if (!o.visible) continue;
            r[0] = o.u; r[1] = o.v; r[2] = o.conA; r[3] = o.conB; r[4] = o.conC;
            r[5] = o.opacity; r[6] = o.rgb[0]; r[7] = o.rgb[1]; r[8] = o.rgb[2]; r[9] = o.t[2];
            radius[s] = o.radius;
            memcpy(rect + 4 * s, o.rect, sizeof o.rect);
            clampmask[s] = o.clampmask;
            /* would a rounding-sized perturbation change the rect? */
            int alt[4];
            double du[2] = {-tol_px, tol_px};
            for (int a = 0; a < 2 && !fragile[s]; a++)
                for (int b2 = 0; b2 < 2 && !fragile[s]; b2++) {
                    tile_rect(o.u + du[a], o.v + du[b2], o.radius, B, Tx, Ty, alt);
                    if (memcmp(alt, o.rect, sizeof alt)) fragile[s] = 1;
                }
            double rtol = 1e-5 * o.r3 + 1e-6;
            if (ceil(o.r3 - rtol) != ceil(o.r3 + rtol)) fragile[s] = 1;
            for (int ch = 0; ch < 3; ch++) {
                /* colour clamp decision near 0 */
                double raw = o.rgb[ch];
                if (!(o.clampmask >> ch & 1) && raw < 1e-6) fragile[s] = 1;
            }
        }
    return 0;
}

/* ------------------------------------------------------------------- binning */

typedef struct { int64_t tile; double z; int64_t slot; } inst_t;

static int inst_cmp(const void *pa, const void *pb)
{
    const inst_t *a = pa, *b = pb;
    if (a->tile != b->tile) return a->tile < b->tile ? -1 : 1;
    if (a->z != b->z) return a->z < b->z ? -1 : 1;
    if (a->slot != b->slot) return a->slot < b->slot ? -1 : 1;
    return 0;
}

/*
 * Tile lists (the binning of the 3DGS renderer the paper keeps, Sec. III-B): every visible
 * slot is listed in each tile of its rect; lists are ordered by (global tile, depth, slot)
 * -- global tile = v*Tx*Ty + ty*Tx + tx, slot = v*n + g, so equal depths keep the
 * Gaussian order (reading).  Depth order is the blending order of Eq. 1.  Inputs are the
 * projected centre, radius and depth of each slot (radius 0 = culled).  Outputs:
 * ranges[2*Ttot] = [start, end) per global tile, the exclusive scan of the per-tile
 * counts (an empty tile is [start, start)), vals[count] = slot ids.  Returns the instance
 * count; writes nothing when that count exceeds `capacity` or vals is NULL (a sizing call).
 */
int64_t orc_bin(const double *u, const double *v, const double *z, const int32_t *radius, int V, int64_t n,
                int W, int H, int B, int64_t capacity, uint32_t *ranges, uint32_t *vals)
{
    int Tx = (W + B - 1) / B, Ty = (H + B - 1) / B;
    int64_t Tv = (int64_t)Tx * Ty;
    /* instances per view: a view's tiles and slots are its own, so views are binned apart */
    int64_t *vcount = calloc((size_t)V + 1, sizeof(int64_t));
#pragma omp parallel for schedule(dynamic)
    for (int vv = 0; vv < V; vv++) {
        int rect[4];
        int64_t c = 0;
        for (int64_t g = 0; g < n; g++) {
            int64_t s = (int64_t)vv * n + g;
            if (radius[s] <= 0) continue;
            tile_rect(u[s], v[s], radius[s], B, Tx, Ty, rect);
            c += (int64_t)(rect[1] - rect[0]) * (rect[3] - rect[2]);
        }
        vcount[vv + 1] = c;
    }
    for (int vv = 0; vv < V; vv++) vcount[vv + 1] += vcount[vv];
    int64_t count = vcount[V];
    if (count > capacity || vals == NULL) {
        free(vcount);
        return count;
    }
#pragma omp parallel for schedule(dynamic)
    for (int vv = 0; vv < V; vv++) {
        int64_t m = vcount[vv + 1] - vcount[vv];
        inst_t *ins = malloc(sizeof(inst_t) * (m ? m : 1));
        int rect[4];
        int64_t k = 0;
        for (int64_t g = 0; g < n; g++) {
            int64_t s = (int64_t)vv * n + g;
            if (radius[s] <= 0) continue;
            tile_rect(u[s], v[s], radius[s], B, Tx, Ty, rect);
            for (int ty = rect[2]; ty < rect[3]; ty++)
                for (int tx = rect[0]; tx < rect[1]; tx++) {
                    ins[k].tile = vv * Tv + (int64_t)ty * Tx + tx;
                    ins[k].z = z[s];
                    ins[k].slot = s;
                    k++;
                }
        }
        qsort(ins, m, sizeof(inst_t), inst_cmp);
        /* ranges: exclusive scan of the per-tile counts (an empty tile is [pos, pos)) */
        int64_t i = 0;
        for (int64_t t = vv * Tv; t < (vv + 1) * Tv; t++) {
            ranges[2 * t] = (uint32_t)(vcount[vv] + i);
            while (i < m && ins[i].tile == t) {
                vals[vcount[vv] + i] = (uint32_t)ins[i].slot;
                i++;
            }
            ranges[2 * t + 1] = (uint32_t)(vcount[vv] + i);
        }
        free(ins);
    }
    free(vcount);
    return count;
}

/* ------------------------------------------------------------- blending (Eq. 1) */

/* Decision codes of one (splat, pixel) step, used for decision hashing. */
enum { D_SKIP_POWER = 1, D_SKIP_ALPHA = 2, D_BLEND = 3, D_BLEND_CLAMPED = 4, D_STOP = 5 };

typedef struct {
    double alpha, T, G, power;
    int64_t slot;
    int clamped;
} step_t;

static uint64_t fnv(uint64_t h, uint64_t x)
{
    for (int i = 0; i < 8; i++) { h ^= (x >> (8 * i)) & 0xff; h *= 1099511628211ULL; }
    return h;
}

/*
 * Front-to-back walk of one pixel along its tile's list (Eq. 1, 3DGS rules):
 *   power = -1/2 (A dx^2 + C dy^2) - B dx dy,  (dx, dy) = (u - x, v - y)
 *   skip if power > 0;  alpha = min(0.99, o exp(power));  skip if alpha < 1/255;
 *   stop before blending a splat if T (1 - alpha) < 1e-4.
 * Records every blended step (alpha, T before it, the Gaussian value G, clamp) in
 * `steps` (if non-NULL).  Returns the number of blended steps; *last = 1-based
 * list position of the last blended splat (0 if none); *Tout = final T;
 * C[3], *D = accumulated colour / depth (without background).
 * `near` reports whether any decision input lay within a relative `tol` of its
 * threshold.
 */
static int walk_pixel(const double *rec, const uint32_t *list, int64_t len, double px, double py,
                      double tol, step_t *steps, double C[3], double *D, double *Tout,
                      uint32_t *last, int *near, uint64_t *hash)
{
    double T = 1.0;
    int nb = 0;
    C[0] = C[1] = C[2] = 0.0;
    *D = 0.0;
    *last = 0;
    *near = 0;
    for (int64_t i = 0; i < len; i++) {
        int64_t s = list[i];
        const double *r = rec + NREC * s;
        double dx = r[0] - px, dy = r[1] - py;
        double power = -0.5 * (r[2] * dx * dx + r[4] * dy * dy) - r[3] * dx * dy;
        if (power > 0.0) {
            if (hash) *hash = fnv(*hash, (uint64_t)i * 8 + D_SKIP_POWER);
            continue;
        }
        double G = exp(power);
        double araw = r[5] * G;
        int clamped = araw > 0.99;
        double alpha = clamped ? 0.99 : araw;
        if (fabs(araw - 0.99) <= tol * 0.99) *near = 1;
        if (fabs(alpha - 1.0 / 255.0) <= tol / 255.0) *near = 1;
        if (alpha < 1.0 / 255.0) {
            if (hash) *hash = fnv(*hash, (uint64_t)i * 8 + D_SKIP_ALPHA);
            continue;
        }
        double testT = T * (1.0 - alpha);
        if (fabs(testT - 1e-4) <= tol * 1e-4) *near = 1;
        if (testT < 1e-4) {
            if (hash) *hash = fnv(*hash, (uint64_t)i * 8 + D_STOP);
            break;
        }
        if (steps) {
            steps[nb].alpha = alpha;
            steps[nb].T = T;
            steps[nb].G = G;
            steps[nb].power = power;
            steps[nb].slot = s;
            steps[nb].clamped = clamped;
        }
        for (int ch = 0; ch < 3; ch++) C[ch] += r[6 + ch] * alpha * T;
        *D += r[9] * alpha * T;
        T = testT;
        nb++;
        *last = (uint32_t)(i + 1);
        if (hash) *hash = fnv(*hash, (uint64_t)i * 8 + (clamped ? D_BLEND_CLAMPED : D_BLEND));
    }
    *Tout = T;
    return nb;
}

/*
 * Forward render of all views and the L1 loss.
 * img[V][3][H][W] = C + T_final * bg; depth[V][H][W] = D (not normalised, reading);
 * T_final, last as in walk_pixel.  If tgt_rgb is non-NULL the per-view loss
 *   L_v = w_v [ mean_{c,x,y} |img - tgt| + lambda_d * mean_{Omega} |depth - tgt_depth| ],
 * Omega = {tgt_depth > 0} (reading), goes to loss_view[v] and |Omega| to depth_count[v].
 * near_px[V][H][W] = 1 where a decision was within `tol` of its threshold.
 * hash (if non-NULL) = a hash of every decision taken, for finite-difference tests.
 */
int orc_render_fwd(const double *rec, const uint32_t *ranges, const uint32_t *vals, int V,
                   int W, int H, int B, const double *bg, const double *cams,
                   const double *tgt_rgb, const double *tgt_depth, double lambda_d, double tol,
                   double *img, double *depth, double *Tfin, uint32_t *last,
                   double *loss_view, int64_t *depth_count, int32_t *near_px, uint64_t *hash)
{
    int Tx = (W + B - 1) / B, Ty = (H + B - 1) / B;
    int64_t HW = (int64_t)H * W;
    if (hash) *hash = 1469598103934665603ULL;
    /* per-row sums of the loss terms, added row after row below */
    double *l1r = calloc((size_t)H, sizeof(double)), *ldr = calloc((size_t)H, sizeof(double));
    int64_t *cntr = calloc((size_t)H, sizeof(int64_t));
    for (int v = 0; v < V; v++) {
        /* the decision hash follows pixel order, so it is formed on one thread */
#pragma omp parallel for schedule(dynamic) if (!hash)
        for (int y = 0; y < H; y++) {
            double l1 = 0.0, ld = 0.0;
            int64_t cnt = 0;
            for (int x = 0; x < W; x++) {
                int64_t tile = (int64_t)v * Tx * Ty + (int64_t)(y / B) * Tx + (x / B);
                uint32_t st = ranges[2 * tile], en = ranges[2 * tile + 1];
                double C[3], D, T;
                uint32_t lst;
                int nr;
                walk_pixel(rec, vals + st, (int64_t)en - st, (double)x, (double)y, tol, NULL,
                           C, &D, &T, &lst, &nr, hash);
                int64_t p = (int64_t)v * HW + (int64_t)y * W + x;
                for (int ch = 0; ch < 3; ch++) img[((int64_t)v * 3 + ch) * HW + (int64_t)y * W + x] = C[ch] + T * bg[ch];
                depth[p] = D;
                Tfin[p] = T;
                last[p] = lst;
                if (near_px) near_px[p] = nr;
                if (tgt_rgb) {
                    for (int ch = 0; ch < 3; ch++) {
                        int64_t q = ((int64_t)v * 3 + ch) * HW + (int64_t)y * W + x;
                        l1 += fabs(img[q] - tgt_rgb[q]);
                    }
                    if (tgt_depth && tgt_depth[p] > 0.0) { ld += fabs(D - tgt_depth[p]); cnt++; }
                }
            }
            l1r[y] = l1;
            ldr[y] = ld;
            cntr[y] = cnt;
        }
        if (tgt_rgb) {
            double l1 = 0.0, ld = 0.0;
            int64_t cnt = 0;
            for (int y = 0; y < H; y++) {
                l1 += l1r[y];
                ld += ldr[y];
                cnt += cntr[y];
            }
            double w = cams[NCAM * v + 16];
            loss_view[v] = w * (l1 / (3.0 * HW) + (cnt > 0 ? lambda_d * ld / cnt : 0.0));
            depth_count[v] = cnt;
        }
    }
    free(l1r);
    free(ldr);
    free(cntr);
    return 0;
}

static double sgn(double x) { return x > 0 ? 1.0 : (x < 0 ? -1.0 : 0.0); }

/*
 * Backward of the blend (Eqs. 2-4): for every pixel, dL/dimg and dL/ddepth from the
 * L1 loss (d|r|/dr = sign(r), 0 at r = 0, reading), or the caller's pixel gradients
 * gimg [V][3][H][W] and gdepth [V][H][W] (NULL: zero) when gimg is non-NULL (the loss
 * of Eq. 9 with its SSIM term); then, for every blended splat k
 * of that pixel (T_k kept from the forward walk, no division):
 *   dI/dc_k = alpha_k T_k,  dD/dz_k = alpha_k T_k
 *   dI/dalpha_k = c_k T_k - (S_k + T_final bg) / (1 - alpha_k),
 *       S_k = sum over splats m blended after k of c_m alpha_m T_m
 *   (same for depth with z and no background)
 *   dalpha/do = G, dalpha/dpower = alpha (both 0 when alpha was clamped at 0.99)
 *   dpower/du = -(A dx + B dy), dpower/dv = -(C dy + B dx),
 *   dpower/dA = -dx^2/2, dpower/dB = -dx dy, dpower/dC = -dy^2/2
 * summed over pixels into grads[V*n][10] (which this function overwrites).  grads_mag
 * (NULL allowed) receives, per field, the sum over pixels of each term evaluated with every
 * operand replaced by its magnitude (|c T| + |colour behind| for the difference in dI/dalpha,
 * |A dx| + |B dy| for dpower/du, ...): the scale that rounding in a lower-precision
 * evaluation of the same terms is proportional to, for tolerance-aware comparisons.  It
 * does not enter grads.
 */
int orc_render_bwd(const double *rec, const uint32_t *ranges, const uint32_t *vals, int V,
                   int64_t n, int W, int H, int B, const double *bg, const double *cams,
                   const double *img, const double *depth, const double *tgt_rgb,
                   const double *tgt_depth, const int64_t *depth_count, double lambda_d,
                   const double *gimg, const double *gdepth, double *grads, double *grads_mag)
{
    int Tx = (W + B - 1) / B, Ty = (H + B - 1) / B;
    int64_t HW = (int64_t)H * W;
    memset(grads, 0, sizeof(double) * NREC * V * n);
    if (grads_mag) memset(grads_mag, 0, sizeof(double) * NREC * V * n);
    int64_t maxlen = 0;
    for (int64_t t = 0; t < (int64_t)V * Tx * Ty; t++) {
        int64_t len = (int64_t)ranges[2 * t + 1] - ranges[2 * t];
        if (len > maxlen) maxlen = len;
    }
    /* views in parallel: the slots a view's pixels write (v*n + g) are that view's own */
#pragma omp parallel for schedule(dynamic)
    for (int v = 0; v < V; v++) {
        step_t *st = malloc(sizeof(step_t) * (maxlen ? maxlen : 1));
        double *S = malloc(sizeof(double) * 4 * (maxlen + 1));
        double w = cams[NCAM * v + 16];
        for (int y = 0; y < H; y++)
            for (int x = 0; x < W; x++) {
                int64_t tile = (int64_t)v * Tx * Ty + (int64_t)(y / B) * Tx + (x / B);
                uint32_t s0 = ranges[2 * tile], s1 = ranges[2 * tile + 1];
                double C[3], D, T;
                uint32_t lst;
                int nr;
                int nb = walk_pixel(rec, vals + s0, (int64_t)s1 - s0, x, y, 0.0, st, C, &D, &T,
                                    &lst, &nr, NULL);
                int64_t p = (int64_t)v * HW + (int64_t)y * W + x;
                double gI[3], gD = 0.0;
                for (int ch = 0; ch < 3; ch++) {
                    int64_t q = ((int64_t)v * 3 + ch) * HW + (int64_t)y * W + x;
                    gI[ch] = gimg ? gimg[q] : w * sgn(img[q] - tgt_rgb[q]) / (3.0 * HW);
                }
                if (gimg)
                    gD = gdepth ? gdepth[p] : 0.0;
                else if (tgt_depth && tgt_depth[p] > 0.0 && depth_count[v] > 0)
                    gD = w * lambda_d * sgn(depth[p] - tgt_depth[p]) / (double)depth_count[v];
                /* suffix sums S_k of contributions behind k */
                for (int j = 0; j < 4; j++) S[4 * nb + j] = 0.0;
                for (int k = nb - 1; k >= 0; k--) {
                    const double *r = rec + NREC * st[k].slot;
                    double wgt = st[k].alpha * st[k].T;
                    for (int ch = 0; ch < 3; ch++) S[4 * k + ch] = S[4 * (k + 1) + ch] + r[6 + ch] * wgt;
                    S[4 * k + 3] = S[4 * (k + 1) + 3] + r[9] * wgt;
                }
                for (int k = 0; k < nb; k++) {
                    const double *r = rec + NREC * st[k].slot;
                    double a = st[k].alpha, Tk = st[k].T;
                    double dLda = 0.0, term[NREC] = {0};
                    double dLda_mag = 0.0, mag[NREC] = {0};   /* magnitudes of the operands */
                    for (int ch = 0; ch < 3; ch++) {
                        double behind = (S[4 * (k + 1) + ch] + T * bg[ch]) / (1.0 - a);
                        double dIda = r[6 + ch] * Tk - behind;
                        dLda += gI[ch] * dIda;
                        dLda_mag += fabs(gI[ch]) * (fabs(r[6 + ch] * Tk) + fabs(behind));
                        term[6 + ch] = gI[ch] * a * Tk;
                        mag[6 + ch] = fabs(term[6 + ch]);
                    }
                    double behind_d = S[4 * (k + 1) + 3] / (1.0 - a);
                    double dDda = r[9] * Tk - behind_d;
                    dLda += gD * dDda;
                    dLda_mag += fabs(gD) * (fabs(r[9] * Tk) + fabs(behind_d));
                    term[9] = gD * a * Tk;
                    mag[9] = fabs(term[9]);
                    if (!st[k].clamped) {
                        double dx = r[0] - x, dy = r[1] - y;
                        double dLdp = dLda * a;              /* dalpha/dpower = alpha */
                        term[5] = dLda * st[k].G;            /* dalpha/do = G */
                        term[0] = dLdp * (-(r[2] * dx + r[3] * dy));
                        term[1] = dLdp * (-(r[4] * dy + r[3] * dx));
                        term[2] = dLdp * (-0.5 * dx * dx);
                        term[3] = dLdp * (-dx * dy);
                        term[4] = dLdp * (-0.5 * dy * dy);
                        double pm = dLda_mag * a;
                        mag[5] = dLda_mag * st[k].G;
                        mag[0] = pm * (fabs(r[2] * dx) + fabs(r[3] * dy));
                        mag[1] = pm * (fabs(r[4] * dy) + fabs(r[3] * dx));
                        mag[2] = pm * 0.5 * dx * dx;
                        mag[3] = pm * fabs(dx * dy);
                        mag[4] = pm * 0.5 * dy * dy;
                    }
                    /* this pixel's contribution (Eq. 4 sums them over the splat's pixels) */
                    double *g = grads + NREC * st[k].slot;
                    for (int f = 0; f < NREC; f++) g[f] += term[f];
                    if (grads_mag) {
                        double *gm = grads_mag + NREC * st[k].slot;
                        for (int f = 0; f < NREC; f++) gm[f] += mag[f];
                    }
                }
            }
        free(st);
        free(S);
    }
    return 0;
}

/* ------------------------------------------------------- preprocess backward */

/*
 * Chain rule from the record derivatives of every visible slot back to the
 * parameters, summed over views.  grads_out has the parameter layout and is
 * overwritten.  Derivations (per slot):
 *   colour: rgb_c = sum_k Y_k(dir) sh_{k,c} + 1/2, clamped at 0 -> dsh = Y g_c (0 where
 *           clamped); ddir = sum_k dY_k sh_k g; dir = d/|d|, d = p - camera centre.
 *   opacity: o = sigmoid(x) -> dx = g_o o (1 - o).
 *   conic Q = Sigma'^{-1}: dL/dSigma' = -Q G_Q Q with G_Q = [[gA, gB/2], [gB/2, gC]].
 *   Sigma' = Tm Sigma Tm^T + 0.3 I, Tm = J Rc: dL/dSigma = Tm^T G Tm, dL/dTm = 2 G Tm Sigma.
 *   J(t): entries fx/tz, fy/tz, -fx x'/tz^2, -fy y'/tz^2 (x' = tx unless guard-band
 *         clamped, where x' = +-lim tz and dx'/dtx = 0, reading).
 *   u = fx tx/tz + cx, v = fy ty/tz + cy, depth = tz, t = Rc p + tc.
 *   Sigma = M M^T, M = R diag(s): dL/dM = 2 (dL/dSigma) M; ds_i = sum_r dM_ri R_ri,
 *   dlog s = ds s; dR_ri = dM_ri s_i; dq = (dqn - qn (qn . dqn)) / |q|.
 */
int orc_preprocess_bwd(const double *P, int64_t n, int deg, const double *cams, int V,
                       int W, int H, int B, double near_z, const double *slot_grads,
                       double *grads_out)
{
    layout_t L = param_layout(n, deg);
    int64_t K = sh_count(deg);
    memset(grads_out, 0, sizeof(double) * L.total);
    for (int v = 0; v < V; v++) {
        const double *cam = cams + NCAM * v;
        const double *Rc = cam;
        double fx = cam[12], fy = cam[13];
        /* Gaussians in parallel: Gaussian g's gradient entries are written by g alone */
#pragma omp parallel for schedule(static)
        for (int64_t g = 0; g < n; g++) {
            proj_t o;
            project(P, n, deg, g, cam, W, H, B, near_z, &o);
            if (!o.visible) continue;
            const double *G = slot_grads + NREC * ((int64_t)v * n + g);
            double dp[3] = {0, 0, 0}, dt[3] = {0, 0, 0};

            /* colour -> SH and direction */
            double gc[3], ddir[3] = {0, 0, 0};
            for (int ch = 0; ch < 3; ch++) gc[ch] = (o.clampmask >> ch & 1) ? 0.0 : G[6 + ch];
            for (int ch = 0; ch < 3; ch++) {
                grads_out[L.dc + 3 * g + ch] += o.Y[0] * gc[ch];
                for (int k = 1; k < K; k++)
                    grads_out[L.rest + 3 * (K - 1) * g + 3 * (k - 1) + ch] += o.Y[k] * gc[ch];
            }
            for (int k = 1; k < K; k++)
                for (int ch = 0; ch < 3; ch++) {
                    double shv = P[L.rest + 3 * (K - 1) * g + 3 * (k - 1) + ch];
                    for (int i = 0; i < 3; i++) ddir[i] += o.dY[k][i] * shv * gc[ch];
                }
            double dd = ddir[0] * o.dir[0] + ddir[1] * o.dir[1] + ddir[2] * o.dir[2];
            for (int i = 0; i < 3; i++) dp[i] += (ddir[i] - o.dir[i] * dd) / o.dnorm;

            /* opacity */
            grads_out[L.opac + g] += G[5] * o.opacity * (1.0 - o.opacity);

            /* conic -> 2D covariance */
            double Q[4] = {o.conA, o.conB, o.conB, o.conC};
            double GQ[4] = {G[2], 0.5 * G[3], 0.5 * G[3], G[4]};
            double tmp[4], Gc[4];
            matmul(Q, GQ, tmp, 2, 2, 2);
            matmul(tmp, Q, Gc, 2, 2, 2);
            for (int i = 0; i < 4; i++) Gc[i] = -Gc[i];

            /* 2D covariance -> Sigma and Tm */
            double Tt[6], GTm[6], GS[9], tmp23[6], tmp32[6];
            transpose(o.Tm, Tt, 2, 3);
            matmul(Tt, Gc, tmp32, 3, 2, 2);
            matmul(tmp32, o.Tm, GS, 3, 2, 3);
            matmul(Gc, o.Tm, tmp23, 2, 2, 3);
            matmul(tmp23, o.Sigma, GTm, 2, 3, 3);
            for (int i = 0; i < 6; i++) GTm[i] *= 2.0;

            /* Tm = J Rc -> J -> t */
            double Rct[9], GJ[6];
            transpose(Rc, Rct, 3, 3);
            matmul(GTm, Rct, GJ, 2, 3, 3);
            double tz = o.t[2], tz2 = tz * tz, tz3 = tz2 * tz;
            dt[2] += GJ[0] * (-fx / tz2) + GJ[4] * (-fy / tz2);
            if (!o.xclamped) {
                dt[0] += GJ[2] * (-fx / tz2);
                dt[2] += GJ[2] * (2.0 * fx * o.t[0] / tz3);
            } else {
                dt[2] += GJ[2] * (fx * o.xsign * o.limx / tz2);
            }
            if (!o.yclamped) {
                dt[1] += GJ[5] * (-fy / tz2);
                dt[2] += GJ[5] * (2.0 * fy * o.t[1] / tz3);
            } else {
                dt[2] += GJ[5] * (fy * o.ysign * o.limy / tz2);
            }
            /* projected centre and depth */
            dt[0] += G[0] * fx / tz;
            dt[2] += -G[0] * fx * o.t[0] / tz2;
            dt[1] += G[1] * fy / tz;
            dt[2] += -G[1] * fy * o.t[1] / tz2;
            dt[2] += G[9];
            for (int i = 0; i < 3; i++) dp[i] += Rc[i] * dt[0] + Rc[3 + i] * dt[1] + Rc[6 + i] * dt[2];
            for (int i = 0; i < 3; i++) grads_out[L.means + 3 * g + i] += dp[i];

            /* Sigma = M M^T -> scale and rotation */
            double GM[9];
            matmul(GS, o.M, GM, 3, 3, 3);
            for (int i = 0; i < 9; i++) GM[i] *= 2.0;
            double GR[9];
            for (int j = 0; j < 3; j++) {
                double ds = 0.0;
                for (int r = 0; r < 3; r++) {
                    ds += GM[3 * r + j] * o.R[3 * r + j];
                    GR[3 * r + j] = GM[3 * r + j] * o.s[j];
                }
                grads_out[L.scales + 3 * g + j] += ds * o.s[j];
            }
            double dR[4][9], dqn[4];
            quat_rot_jac(o.qn, dR);
            for (int k = 0; k < 4; k++) {
                dqn[k] = 0.0;
                for (int i = 0; i < 9; i++) dqn[k] += GR[i] * dR[k][i];
            }
            double proj = dqn[0] * o.qn[0] + dqn[1] * o.qn[1] + dqn[2] * o.qn[2] + dqn[3] * o.qn[3];
            for (int k = 0; k < 4; k++) grads_out[L.quats + 4 * g + k] += (dqn[k] - o.qn[k] * proj) / o.qnorm;
        }
    }
    return 0;
}

/* ------------------------------------------------------------ densify stats */

/*
 * Per visible slot (radius > 0): accum[g] += || (dL_v/du * W/2, dL_v/dv * H/2) ||
 * (gradient of this view's loss w.r.t. the projected centre, in NDC units, reading),
 * denom[g] += 1, max_r2d[g] = max(max_r2d[g], radius).  Accumulates into the outputs.
 */
int orc_densify_stats(const double *slot_grads, const int32_t *radius, int V, int64_t n, int W, int H,
                      double *accum, double *denom, double *max_r2d)
{
    for (int v = 0; v < V; v++)
        for (int64_t g = 0; g < n; g++) {
            int64_t s = (int64_t)v * n + g;
            if (radius[s] <= 0) continue;
            double gx = slot_grads[NREC * s] * 0.5 * W, gy = slot_grads[NREC * s + 1] * 0.5 * H;
            accum[g] += sqrt(gx * gx + gy * gy);
            denom[g] += 1.0;
            if (radius[s] > max_r2d[g]) max_r2d[g] = radius[s];
        }
    return 0;
}

/*
 * Forward blend (Eq. 1) of a list of pixels only: pix[k] = (view, x, y); writes
 * img[k][3] (with background), depth[k], T[k], last[k] and a near-threshold flag.
 * For sampled comparisons on workloads too large to render in full.
 */
int orc_render_pixels(const double *rec, const uint32_t *ranges, const uint32_t *vals, int W, int H, int B,
                      const double *bg, const int32_t *pix, int64_t npix, double tol, double *img, double *depth,
                      double *Tfin, uint32_t *last, int32_t *near_px)
{
    int Tx = (W + B - 1) / B, Ty = (H + B - 1) / B;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < npix; k++) {
        int v = pix[3 * k], x = pix[3 * k + 1], y = pix[3 * k + 2];
        int64_t tile = (int64_t)v * Tx * Ty + (int64_t)(y / B) * Tx + (x / B);
        uint32_t st = ranges[2 * tile], en = ranges[2 * tile + 1];
        double C[3], D, T;
        uint32_t lst;
        int nr;
        walk_pixel(rec, vals + st, (int64_t)en - st, (double)x, (double)y, tol, NULL, C, &D, &T, &lst, &nr, NULL);
        for (int ch = 0; ch < 3; ch++) img[3 * k + ch] = C[ch] + T * bg[ch];
        depth[k] = D;
        Tfin[k] = T;
        last[k] = lst;
        near_px[k] = nr;
    }
    return 0;
}

/*
 * Geometric densification (Sec. III-A.3, III-B: a keyframe's coloured point cloud becomes
 * initial Gaussians, initialised as in 3DGS).  For every point i, the mean squared distance
 * to its k nearest other points, by brute force over all pairs: out[i] = (1/k') sum of the
 * k' = min(k, m - 1) smallest |x_i - x_j|^2, j != i (0 when m = 1).  Duplicated points are
 * neighbours at distance 0.
 */
static double knn_one(const double *xyz, int64_t m, int k, int64_t i)
{
    double best[16];
    int nb = 0;
    for (int64_t j = 0; j < m; j++) {
        if (j == i) continue;
        double dx = xyz[3 * j] - xyz[3 * i], dy = xyz[3 * j + 1] - xyz[3 * i + 1],
               dz = xyz[3 * j + 2] - xyz[3 * i + 2];
        double d = dx * dx + dy * dy + dz * dz;
        /* keep the nb smallest, ascending */
        if (nb < k) {
            best[nb++] = d;
        } else if (d < best[k - 1]) {
            best[k - 1] = d;
        } else {
            continue;
        }
        for (int a = nb - 1; a > 0 && best[a] < best[a - 1]; a--) {
            double t = best[a];
            best[a] = best[a - 1];
            best[a - 1] = t;
        }
    }
    double s = 0.0;
    for (int a = 0; a < nb; a++) s += best[a];
    return nb ? s / nb : 0.0;
}

int orc_knn_mean_d2(const double *xyz, int64_t m, int k, double *out)
{
    if (k < 1 || k > 16) return -1;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < m; i++) out[i] = knn_one(xyz, m, k, i);
    return 0;
}

/* The same for the listed points only (idx[s]), for sampled checks of large clouds. */
int orc_knn_mean_d2_at(const double *xyz, int64_t m, int k, const int64_t *idx, int64_t s, double *out)
{
    if (k < 1 || k > 16) return -1;
    for (int64_t t = 0; t < s; t++)
        if (idx[t] < 0 || idx[t] >= m) return -2;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < s; t++) out[t] = knn_one(xyz, m, k, idx[t]);
    return 0;
}
