/* FP64 CPU oracle of the NeDF composition render path (arXiv 2308.04669).
 *
 * TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference leg may load this.  It is deliberately plain: nested loops in the order of the
 * paper's Algorithm 1 (Steps 1-2) and Algorithm 2 (Step 3), every quantity in double.
 *
 * Readings of points the paper leaves open are stated where they are used; each one is also
 * listed in the repository's design notes.
 */
#include "nedf_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define PI 3.14159265358979323846

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double len3(const double *a) { return sqrt(dot3(a, a)); }
static double dmin(double a, double b) { return a < b ? a : b; }
static double dmax(double a, double b) { return a > b ? a : b; }
static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }
static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static void normalize3(double *a)
{
    double l = len3(a);
    a[0] /= l; a[1] /= l; a[2] /= l;
}

/* ------------------------------------------------------------------------------------------ */
/* Analytic shapes (object-local).  These stand in for the pre-trained NeRF objects.            */
/* ------------------------------------------------------------------------------------------ */
static double sdf_torus_y(double x, double y, double z, double R, double r)
{
    double q0 = sqrt(x * x + z * z) - R;
    return sqrt(q0 * q0 + y * y) - r;
}

double orc_sdf(int kind, const double *p, const double x[3])
{
    switch (kind) {
    case ORC_SPHERE:
        return len3(x) - p[0];
    case ORC_TORUS:
        return sdf_torus_y(x[0], x[1], x[2], p[0], p[1]);
    case ORC_BOX: {
        double q[3], outside = 0.0, inside;
        for (int c = 0; c < 3; ++c) q[c] = fabs(x[c]) - p[c];
        for (int c = 0; c < 3; ++c) outside += dmax(q[c], 0.0) * dmax(q[c], 0.0);
        inside = dmin(dmax(q[0], dmax(q[1], q[2])), 0.0);
        return sqrt(outside) + inside;
    }
    case ORC_CAPSULE: { /* segment on the y axis, |y| <= p0, radius p1 */
        double y = x[1] - clampd(x[1], -p[0], p[0]);
        return sqrt(x[0] * x[0] + y * y + x[2] * x[2]) - p[1];
    }
    case ORC_ROUNDCONE: {
        /* Convex hull of sphere (0,y1,0) radius r1 and sphere (0,y2,0) radius r2, reduced to the
         * half-plane (radial distance, height): distance to the hull of two discs. */
        double r1 = p[0], y1 = p[1], r2 = p[2], y2 = p[3];
        double h = y2 - y1;
        double qr = sqrt(x[0] * x[0] + x[2] * x[2]), qy = x[1] - y1;
        double sb = (r1 - r2) / h;           /* sine of the side's tilt */
        double cb = sqrt(1.0 - sb * sb);     /* cosine of the side's tilt */
        double k = -qr * sb + qy * cb;       /* position along the side's tangent direction */
        if (k < 0.0) return sqrt(qr * qr + qy * qy) - r1;
        if (k > cb * h) return sqrt(qr * qr + (qy - h) * (qy - h)) - r2;
        return qr * cb + qy * sb - r1;
    }
    case ORC_TWOSPHERE: {
        double a[3] = {x[0] - p[0], x[1], x[2]}, b[3] = {x[0] + p[0], x[1], x[2]};
        return dmin(len3(a), len3(b)) - p[1];
    }
    case ORC_TWISTTORUS: { /* ring in the xy plane (axis z), twisted about y by p2 rad per unit y */
        double th = p[2] * x[1], c = cos(th), s = sin(th);
        double xr = c * x[0] - s * x[2], zr = s * x[0] + c * x[2];
        double q0 = sqrt(xr * xr + x[1] * x[1]) - p[0];
        return sqrt(q0 * q0 + zr * zr) - p[1];
    }
    case ORC_OCTA: /* |x|+|y|+|z| = a, scaled to a lower bound of the distance */
        return (fabs(x[0]) + fabs(x[1]) + fabs(x[2]) - p[0]) / sqrt(3.0);
    default:
        return 1e30;
    }
}

/* sigma(x) = sigma_max * sigmoid(-sdf / width): the analytic NeRF density of the workloads. */
double orc_density(const orc_scene *sc, int type, const double x[3])
{
    const orc_type *t = &sc->types[type];
    return sc->sigma_max / (1.0 + exp(orc_sdf(t->kind, t->params, x) / sc->sdf_width));
}

static int inside_solid(const orc_scene *sc, int type, const double x[3])
{
    /* The iso level sigma_max / 2 (reading: surface = half of the peak density). */
    return orc_density(sc, type, x) >= 0.5 * sc->sigma_max;
}

/* ------------------------------------------------------------------------------------------ */
/* Step 1 inputs: camera rays, rigid transform of rays (Eq. 7), bound cull (Fig. 2b)            */
/* ------------------------------------------------------------------------------------------ */
void orc_camera_ray(const orc_scene *sc, int i, int j, double o[3], double d[3])
{
    double fwd[3] = {sc->target[0] - sc->eye[0], sc->target[1] - sc->eye[1], sc->target[2] - sc->eye[2]};
    double up0[3] = {0.0, 1.0, 0.0}, right[3], up[3];
    normalize3(fwd);
    cross3(fwd, up0, right);
    normalize3(right);
    cross3(right, fwd, up);
    double th = tan(0.5 * sc->fov_deg * PI / 180.0);
    double u = (2.0 * (i + 0.5) / sc->W - 1.0) * th * ((double)sc->W / sc->H);
    double v = (1.0 - 2.0 * (j + 0.5) / sc->H) * th;
    for (int c = 0; c < 3; ++c) {
        o[c] = sc->eye[c];
        d[c] = u * right[c] + v * up[c] + fwd[c];
    }
    normalize3(d);
}

/* G^{-1}: local origin R^T (o - T) / s, local direction R^T d / s normalised (the local ray
 * parameter times s is the world distance). */
void orc_to_local(const orc_scene *sc, int inst, const double o[3], const double d[3],
                  double ol[3], double dl[3])
{
    const double *R = sc->inst_R + 9 * inst, *T = sc->inst_T + 3 * inst;
    double s = sc->inst_s[inst];
    double v[3] = {o[0] - T[0], o[1] - T[1], o[2] - T[2]};
    for (int c = 0; c < 3; ++c) {
        ol[c] = (R[0 * 3 + c] * v[0] + R[1 * 3 + c] * v[1] + R[2 * 3 + c] * v[2]) / s;
        dl[c] = (R[0 * 3 + c] * d[0] + R[1 * 3 + c] * d[1] + R[2 * 3 + c] * d[2]) / s;
    }
    normalize3(dl);
}

/* Ray vs the bound sphere |x| = rb.  Kept iff the ray meets the sphere ahead of its origin.
 * out4 = {t_entry (clamped at 0), t_exit, t_perp, discriminant}.  t_perp = -o.d is the signed
 * distance from the origin to the tangency point p_perp of Eq. 2 (Fig. 2a). */
int orc_bound(const double ol[3], const double dl[3], double rb, double out4[4])
{
    double b = dot3(ol, dl);
    double c = dot3(ol, ol) - rb * rb;
    double disc = b * b - c;
    out4[0] = INFINITY;
    out4[1] = -INFINITY;
    out4[2] = -b;
    out4[3] = disc;
    if (disc < 0.0) return 0;
    double sq = sqrt(disc);
    out4[1] = -b + sq;
    out4[0] = dmax(0.0, -b - sq);
    return out4[1] >= 0.0;
}

/* gamma(x) = [x, sin(2^0 x) .. sin(2^{L-1} x), cos(2^0 x) .. cos(2^{L-1} x)], blocks n wide. */
int orc_posenc(const double *x, int n, int L, double *out)
{
    for (int c = 0; c < n; ++c) out[c] = x[c];
    for (int k = 0; k < L; ++k)
        for (int c = 0; c < n; ++c) {
            out[n + k * n + c] = sin(ldexp(x[c], k));
            out[n + L * n + k * n + c] = cos(ldexp(x[c], k));
        }
    return n * (1 + 2 * L);
}

/* NeDF input: the ray's entry point on the bound plus its direction, encoded with 6
 * frequencies (78 features). */
int orc_nedf_features(const double ol[3], const double dl[3], double rb, double *feat, double out4[4])
{
    if (!orc_bound(ol, dl, rb, out4)) return 0;
    double x[6];
    for (int c = 0; c < 3; ++c) {
        x[c] = ol[c] + out4[0] * dl[c];
        x[3 + c] = dl[c];
    }
    orc_posenc(x, 6, 6, feat);
    return 1;
}

/* ------------------------------------------------------------------------------------------ */
/* Networks                                                                                    */
/* ------------------------------------------------------------------------------------------ */
double orc_round_bf16(double x)
{
    /* Round to the nearest value with an 8-bit significand, ties to even. */
    if (x == 0.0 || !isfinite(x)) return x;
    int e;
    frexp(x, &e); /* |x| in [2^(e-1), 2^e) */
    double q = ldexp(1.0, e - 8);
    return nearbyint(x / q) * q;
}

double orc_round_e4m3(double x)
{
    /* OCP FP8 E4M3 (no infinities): 3 fraction bits, exponent bias 7, normals from 2^-6, subnormal
     * spacing 2^-9, largest finite 448.  Nearest value, ties to even; beyond 448 saturates to 448. */
    if (x == 0.0 || isnan(x)) return x;
    int e;
    frexp(x, &e);                                   /* |x| in [2^(e-1), 2^e) */
    int ulp_exp = e - 1 - 3;                        /* spacing of 4-bit significands in that binade */
    if (ulp_exp < -9) ulp_exp = -9;                 /* subnormal range keeps the 2^-9 spacing */
    double q = ldexp(nearbyint(ldexp(x, -ulp_exp)), ulp_exp);
    if (q > 448.0) q = 448.0;
    if (q < -448.0) q = -448.0;
    return q;
}

double orc_fp8_scale(double max_abs)
{
    /* The power of two s with max_abs / s in (224, 448]; 1 for an all-zero layer. */
    if (!(max_abs > 0.0)) return 1.0;
    int e;
    frexp(max_abs / 448.0, &e);                     /* max_abs / 448 in [2^(e-1), 2^e) */
    double s = ldexp(1.0, e);
    if (max_abs / ldexp(1.0, e - 1) <= 448.0) s = ldexp(1.0, e - 1);   /* exact power of two */
    return s;
}

/* Distance from v to the nearest rounding boundary of the BF16 (fmt 0) or E4M3 (fmt 1) grid: how
 * far v may move before it rounds to another value.  Zero stays zero.  Boundaries are the
 * midpoints between neighbouring representable values; below a binade's first value the grid is
 * twice as fine (except below E4M3's smallest normal), hence the second candidate.  E4M3 saturates at 448, so the last boundary is 432. */
double orc_round_margin(double v, int fmt)
{
    double a = fabs(v);
    if (a == 0.0 || !isfinite(a)) return INFINITY;
    if (fmt == 1 && a >= 448.0) return a - 432.0;
    int e;
    frexp(a, &e);                                   /* a in [2^(e-1), 2^e) */
    int qe = fmt == 0 ? e - 8 : e - 1 - 3;
    int sub = fmt == 1 && qe < -9;
    if (sub) qe = -9;
    double q = ldexp(1.0, qe), u = a / q;
    double m = fabs(u - floor(u) - 0.5) * q;
    if (!sub && !(fmt == 1 && qe == -9)) m = dmin(m, a - ldexp(1.0, e - 1) + 0.25 * q);   /* E4M3's subnormals
                                                        keep the smallest normal binade's spacing */
    return m;
}

/* Rounds v to BF16 (fmt 0) or E4M3 (fmt 1); with `flip` set, to the representable value on the
 * other side of v's nearest rounding boundary instead (the value a slightly different sum of the
 * same terms would have rounded to). */
static double round_fmt(double v, int fmt, int flip)
{
    double q = fmt == 0 ? orc_round_bf16(v) : orc_round_e4m3(v);
    if (!flip) return q;
    double m = orc_round_margin(v, fmt);
    if (!isfinite(m)) return q;
    double step = m * (1.0 + 1e-9) + 1e-300;
    double up = fmt == 0 ? orc_round_bf16(v + step) : orc_round_e4m3(v + step);
    double dn = fmt == 0 ? orc_round_bf16(v - step) : orc_round_e4m3(v - step);
    return up != q ? up : dn;
}

/* The MLP of readings 20/21 with rounding diagnostics.  Every BF16 / E4M3-rounded value has an
 * index: the input features 0 .. dims[0]-1, then each hidden layer's outputs in order.
 *   qmargin   (may be NULL) the row's smallest distance of a rounded value to its rounding
 *             boundary, relative to the scale that bounds another implementation's error there
 *             (sum of |w a| plus |b| for a layer's output, max(|v|, 1/4) for an input feature);
 *   flips     the indices of the n_flips values rounded to their other neighbour;
 *   n_cand    the n_cand values of smallest relative margin are listed in cand_idx / cand_margin
 *             (ascending; unused entries get index -1). */
static int in_flips(int vidx, int n_flips, const int *flips)
{
    for (int k = 0; k < n_flips; ++k)
        if (flips[k] == vidx) return 1;
    return 0;
}

static void mlp_core_set(const double *w, int n_layers, const int *dims, const double *x, double *y, int quant,
                         double *qmargin, int n_flips, const int *flips, int n_cand, int *cand_idx, double *cand_margin)
{
    int maxd = 0;
    for (int l = 0; l <= n_layers; ++l) maxd = dims[l] > maxd ? dims[l] : maxd;
    double *a = (double *)malloc(sizeof(double) * maxd), *b = (double *)malloc(sizeof(double) * maxd);
    for (int c = 0; c < n_cand; ++c) { cand_idx[c] = -1; cand_margin[c] = INFINITY; }
    double qm = INFINITY;
    int vidx = 0;
    /* records value index vidx with relative margin r among the smallest n_cand */
#define NOTE_MARGIN(r)                                                                     \
    do {                                                                                   \
        double r_ = (r);                                                                   \
        qm = dmin(qm, r_);                                                                 \
        if (n_cand > 0 && r_ < cand_margin[n_cand - 1]) {                                  \
            int c_ = n_cand - 1;                                                           \
            while (c_ > 0 && cand_margin[c_ - 1] > r_) {                                   \
                cand_margin[c_] = cand_margin[c_ - 1]; cand_idx[c_] = cand_idx[c_ - 1]; --c_; \
            }                                                                              \
            cand_margin[c_] = r_; cand_idx[c_] = vidx;                                     \
        }                                                                                  \
    } while (0)
    for (int i = 0; i < dims[0]; ++i, ++vidx) {
        a[i] = x[i];
        if (quant == ORC_QUANT_NONE) continue;
        /* an input feature (a coordinate, or the sine or cosine of one scaled by up to 2^9) carries
         * an absolute error from the coordinates: its margin is measured against |v| but no less
         * than 1/4 */
        NOTE_MARGIN(orc_round_margin(x[i], 0) / dmax(fabs(x[i]), 0.25));
        a[i] = round_fmt(x[i], 0, in_flips(vidx, n_flips, flips));
    }
    const double *p = w;
    for (int l = 0; l < n_layers; ++l) {
        int fi = dims[l], fo = dims[l + 1];
        const double *W = p, *bias = p + (size_t)fi * fo;
        /* FP8 mode: hidden-to-hidden layers (not the first, not the output layer) in E4M3 */
        const int fp8_layer = quant == ORC_QUANT_FP8 && l > 0 && l + 1 < n_layers;
        double s = 1.0;
        if (fp8_layer) {
            double m = 0.0;
            for (size_t i = 0; i < (size_t)fi * fo; ++i) m = dmax(m, fabs(W[i]));
            s = orc_fp8_scale(m);
        }
        for (int o = 0; o < fo; ++o) {
            double acc = 0.0, mag = 0.0;
            for (int i = 0; i < fi; ++i) {
                double wv = W[(size_t)o * fi + i], av = a[i];
                if (quant == ORC_QUANT_BF16) wv = orc_round_bf16(wv);
                else if (quant == ORC_QUANT_FP8) wv = fp8_layer ? s * orc_round_e4m3(wv / s) : orc_round_bf16(wv);
                acc += wv * av;
                mag += fabs(wv * av);
            }
            /* reading 20: a layer whose products take BF16 operands (every hidden layer in the BF16
             * mode, the first in the FP8 mode) takes its bias as the sum of two BF16 values, the
             * rounded bias and the rounded remainder (16 significant bits); the output layer and
             * the E4M3 layers add it in full */
            double bv = bias[o];
            if (l + 1 < n_layers && (quant == ORC_QUANT_BF16 || (quant == ORC_QUANT_FP8 && l == 0))) {
                const double hi = orc_round_bf16(bv);
                bv = hi + orc_round_bf16(bv - hi);
            }
            acc += bv;
            mag += fabs(bv);
            b[o] = (l + 1 < n_layers) ? dmax(acc, 0.0) : acc;
            if (quant != ORC_QUANT_NONE && l + 1 < n_layers) {
                /* hidden activations: BF16, or E4M3 in the FP8 mode (they feed E4M3 layers) */
                int fmt = quant == ORC_QUANT_FP8 ? 1 : 0;
                NOTE_MARGIN(orc_round_margin(b[o], fmt) / dmax(mag, 1e-300));
                b[o] = round_fmt(b[o], fmt, in_flips(vidx, n_flips, flips));
                ++vidx;
            }
        }
        memcpy(a, b, sizeof(double) * fo);
        p += (size_t)fi * fo + fo;
    }
#undef NOTE_MARGIN
    memcpy(y, a, sizeof(double) * dims[n_layers]);
    if (qmargin) *qmargin = qm;
    free(a);
    free(b);
}

static void mlp_core2(const double *w, int n_layers, const int *dims, const double *x, double *y, int quant,
                      double *qmargin, int flip_idx, int flip_idx2, int n_cand, int *cand_idx, double *cand_margin)
{
    const int flips[2] = {flip_idx, flip_idx2};
    mlp_core_set(w, n_layers, dims, x, y, quant, qmargin, 2, flips, n_cand, cand_idx, cand_margin);
}

static void mlp_core(const double *w, int n_layers, const int *dims, const double *x, double *y, int quant,
                     double *qmargin, int flip_idx, int n_cand, int *cand_idx, double *cand_margin)
{
    mlp_core2(w, n_layers, dims, x, y, quant, qmargin, flip_idx, -1, n_cand, cand_idx, cand_margin);
}

void orc_mlp(const double *w, int n_layers, const int *dims, const double *x, double *y, int quant)
{
    mlp_core(w, n_layers, dims, x, y, quant, NULL, -1, 0, NULL, NULL);
}

double orc_mlp_qmargin(const double *w, int n_layers, const int *dims, const double *x, double *y, int quant)
{
    double qm;
    mlp_core(w, n_layers, dims, x, y, quant, &qm, -1, 0, NULL, NULL);
    return qm;
}

void orc_mlp_flip(const double *w, int n_layers, const int *dims, const double *x, double *y, int quant,
                  int flip_idx, int n_cand, int *cand_idx, double *cand_margin)
{
    mlp_core(w, n_layers, dims, x, y, quant, NULL, flip_idx, n_cand, cand_idx, cand_margin);
}

void orc_mlp_flip2(const double *w, int n_layers, const int *dims, const double *x, double *y, int quant, int flip_a,
                   int flip_b)
{
    mlp_core2(w, n_layers, dims, x, y, quant, NULL, flip_a, flip_b, 0, NULL, NULL);
}

void orc_mlp_flipset(const double *w, int n_layers, const int *dims, const double *x, double *y, int quant,
                     int n_flips, const int *flips)
{
    mlp_core_set(w, n_layers, dims, x, y, quant, NULL, n_flips, flips, 0, NULL, NULL);
}

static int nedf_dims(const orc_type *t, int *dims)
{
    dims[0] = 78;
    for (int l = 1; l <= t->nedf_hidden; ++l) dims[l] = t->nedf_width;
    dims[t->nedf_hidden + 1] = 2;
    return t->nedf_hidden + 1;
}

static int nerf_dims(const orc_type *t, int *dims)
{
    dims[0] = 90;
    for (int l = 1; l <= t->nerf_hidden; ++l) dims[l] = t->nerf_width;
    dims[t->nerf_hidden + 1] = 3;
    return t->nerf_hidden + 1;
}

/* ------------------------------------------------------------------------------------------ */
/* The paper's intersection network (Section "Intersection network", Eq. 3-4 and 6, Appendix A) */
/* ------------------------------------------------------------------------------------------ */
/* Offsets into the packed weights (W[out][in] then b[out], layer after layer). */
static size_t cls_block_off(int k) { return (size_t)ORC_CLS_IN * ORC_CLS_W + ORC_CLS_W + (size_t)k * 2 * (ORC_CLS_W * ORC_CLS_W + ORC_CLS_W); }
static size_t cls_tail_off(void) { return cls_block_off(ORC_CLS_BLOCKS); }

int64_t orc_cls_param_count(void)
{
    return (int64_t)cls_tail_off() + (int64_t)(1 + ORC_CLS_NC) * (ORC_CLS_W + 1) + (int64_t)ORC_CLS_NF * (ORC_CLS_W + 1);
}

/* Input (Section "NeDF": a ray is represented by 16 points sampled within a local range along it;
 * reading: uniform over the chord [t_e, t_x] through the bound sphere, both ends included), each
 * point encoded as in NeRF with 10 frequencies: [p, sin(2^k p), cos(2^k p)], 63 values. */
int orc_cls_features(const double ol[3], const double dl[3], double rb, double *feat, double out4[4])
{
    if (!orc_bound(ol, dl, rb, out4)) return 0;
    for (int j = 0; j < ORC_CLS_PTS; ++j) {
        const double t = out4[0] + (out4[1] - out4[0]) * j / (ORC_CLS_PTS - 1);
        double p[3];
        for (int c = 0; c < 3; ++c) p[c] = ol[c] + t * dl[c];
        orc_posenc(p, 3, ORC_CLS_FREQ, feat + 63 * j);
    }
    return 1;
}

/* The BF16 copy of the weights: every matrix entry rounded, biases kept. */
void orc_cls_round_bf16(const double *w, double *wq)
{
    const int64_t n = orc_cls_param_count();
    for (int64_t i = 0; i < n; ++i) wq[i] = w[i];
    const int fi[4] = {ORC_CLS_IN, ORC_CLS_W, ORC_CLS_W, ORC_CLS_W};
    size_t off = 0;
    /* head, then 32 body layers, then the two tails: round W, skip b */
    for (int l = 0; l < 1 + 2 * ORC_CLS_BLOCKS + 2; ++l) {
        const int in = l == 0 ? fi[0] : ORC_CLS_W;
        const int out = l < 1 + 2 * ORC_CLS_BLOCKS ? ORC_CLS_W : (l == 1 + 2 * ORC_CLS_BLOCKS ? 1 + ORC_CLS_NC : ORC_CLS_NF);
        for (size_t i = 0; i < (size_t)in * out; ++i) wq[off + i] = orc_round_bf16(w[off + i]);
        off += (size_t)in * out + out;
    }
}

/* y = W x + b for one packed layer */
static void cls_affine(const double *W, int fi, int fo, const double *x, double *y)
{
    const double *b = W + (size_t)fi * fo;
    for (int o = 0; o < fo; ++o) {
        const double *row = W + (size_t)o * fi;
        double acc = 0.0;
        for (int i = 0; i < fi; ++i) acc += row[i] * x[i];
        y[o] = acc + b[o];
    }
}

static double cls_q(double v, int quant) { return quant == ORC_QUANT_NONE ? v : orc_round_bf16(v); }

/* Forward pass, saving what the backward pass needs (any pointer may be NULL):
 *   h[k] (k = 0..16): the input of block k (h[16] feeds the tails), u[k] = W1 h + b1,
 *   z[k] = h + W2 ReLU(u) + b2.
 * Head: a single linear layer.  Residual block (reading of "two fully connected layers followed
 * by ReLU" with a skip connection, as in He et al.'s basic block): h' = ReLU(h + W2 ReLU(W1 h + b1)
 * + b2).  Tails: linear.  quant BF16 (or FP8, which the classifier runs as BF16): the network input
 * and every layer's input rounded to BF16 (weights come pre-rounded in w); sums and biases in
 * double. */
static void cls_forward_saved(const double *w, const double *x, double *logits, int quant, double *hs, double *us,
                              double *zs)
{
    double xin[ORC_CLS_IN], h[ORC_CLS_W], u[ORC_CLS_W], t[ORC_CLS_W], z[ORC_CLS_W];
    for (int i = 0; i < ORC_CLS_IN; ++i) xin[i] = cls_q(x[i], quant);
    cls_affine(w, ORC_CLS_IN, ORC_CLS_W, xin, h);
    for (int i = 0; i < ORC_CLS_W; ++i) h[i] = cls_q(h[i], quant);
    for (int k = 0; k < ORC_CLS_BLOCKS; ++k) {
        const double *W1 = w + cls_block_off(k), *W2 = W1 + ORC_CLS_W * ORC_CLS_W + ORC_CLS_W;
        if (hs) memcpy(hs + (size_t)k * ORC_CLS_W, h, sizeof(h));
        cls_affine(W1, ORC_CLS_W, ORC_CLS_W, h, u);
        for (int i = 0; i < ORC_CLS_W; ++i) t[i] = cls_q(dmax(u[i], 0.0), quant);
        cls_affine(W2, ORC_CLS_W, ORC_CLS_W, t, z);
        for (int i = 0; i < ORC_CLS_W; ++i) z[i] += h[i];
        if (us) memcpy(us + (size_t)k * ORC_CLS_W, u, sizeof(u));
        if (zs) memcpy(zs + (size_t)k * ORC_CLS_W, z, sizeof(z));
        for (int i = 0; i < ORC_CLS_W; ++i) h[i] = cls_q(dmax(z[i], 0.0), quant);
    }
    if (hs) memcpy(hs + (size_t)ORC_CLS_BLOCKS * ORC_CLS_W, h, sizeof(h));
    const double *TA = w + cls_tail_off(), *TB = TA + (size_t)(1 + ORC_CLS_NC) * (ORC_CLS_W + 1);
    cls_affine(TA, ORC_CLS_W, 1 + ORC_CLS_NC, h, logits);
    cls_affine(TB, ORC_CLS_W, ORC_CLS_NF, h, logits + 1 + ORC_CLS_NC);
}

void orc_cls_forward(const double *w, const double *x, double *logits, int quant)
{
    cls_forward_saved(w, x, logits, quant, NULL, NULL, NULL);
}

/* Segment operator S (Section "Intersection network"): m = mu / l in [-1, 1] to the coarse bin c
 * of N_c over [-1, 1] and the fine bin f of N_f inside it. */
void orc_cls_segment(double m, int *c, int *f)
{
    const double u = (m + 1.0) * 0.5 * ORC_CLS_NC;      /* coarse position in bins */
    int cc = (int)floor(u);
    cc = cc < 0 ? 0 : (cc >= ORC_CLS_NC ? ORC_CLS_NC - 1 : cc);
    int ff = (int)floor((u - cc) * ORC_CLS_NF);
    ff = ff < 0 ? 0 : (ff >= ORC_CLS_NF ? ORC_CLS_NF - 1 : ff);
    *c = cc;
    *f = ff;
}

/* Eq. 4: mu = 2l argmax(v_c) / N_c + (2l / N_c) argmax(v_f) / N_f - l, returned as m = mu / l;
 * a = the hit logit.  Returns the smaller of the two top-2 logit gaps (how far the argmax
 * decisions are from a tie); the first maximum wins a tie. */
double orc_cls_decode(const double *logits, double *m, double *a, int *c, int *f)
{
    double gap = INFINITY;
    int best[2];
    const int base[2] = {1, 1 + ORC_CLS_NC}, nb[2] = {ORC_CLS_NC, ORC_CLS_NF};
    for (int s = 0; s < 2; ++s) {
        int bi = 0;
        double b1 = -INFINITY, b2 = -INFINITY;
        for (int i = 0; i < nb[s]; ++i) {
            const double v = logits[base[s] + i];
            if (v > b1) { b2 = b1; b1 = v; bi = i; }
            else if (v > b2) b2 = v;
        }
        best[s] = bi;
        gap = dmin(gap, b1 - b2);
    }
    *c = best[0];
    *f = best[1];
    *m = 2.0 * best[0] / ORC_CLS_NC + (2.0 / ORC_CLS_NC) * best[1] / ORC_CLS_NF - 1.0;
    *a = logits[0];
    return gap;
}

static double bce_logit(double x, double y) { return dmax(x, 0.0) - x * y + log1p(exp(-fabs(x))); }

/* Eq. 6 for a batch of n rays given as network inputs x[n][1008] with labels (m*, hit*):
 *   L = mean over labelled hits of [BCE(v_c, onehot S_c(m*)) + BCE(v_f, onehot S_f(m*))]
 *       + 0.1 * mean over all rays of BCE(a, hit*),
 * each BCE the mean over its bins of the logistic cross-entropy (reading: the bin terms are
 * defined only where the ray hits).  grad receives dL/dtheta in the packed layout (double
 * arithmetic, no rounding).  Returns L. */
double orc_cls_loss_grad(const double *w, int n, const double *x, const double *m_star, const int *hit_star,
                         double *grad)
{
    const int64_t np = orc_cls_param_count();
    memset(grad, 0, sizeof(double) * np);
    const size_t HW = (size_t)(ORC_CLS_BLOCKS + 1) * ORC_CLS_W;
    double *hs = (double *)malloc(sizeof(double) * HW), *us = (double *)malloc(sizeof(double) * HW);
    double *zs = (double *)malloc(sizeof(double) * HW);
    double logits[ORC_CLS_OUT], g[ORC_CLS_OUT], dh[ORC_CLS_W], dz[ORC_CLS_W], dt[ORC_CLS_W], du[ORC_CLS_W];
    int n_hit = 0;
    for (int k = 0; k < n; ++k) n_hit += hit_star[k] != 0;
    double loss = 0.0;
    for (int r = 0; r < n; ++r) {
        const double *xr = x + (size_t)r * ORC_CLS_IN;
        cls_forward_saved(w, xr, logits, ORC_QUANT_NONE, hs, us, zs);
        const double al = hit_star[r] ? 1.0 : 0.0;
        loss += 0.1 * bce_logit(logits[0], al) / n;
        g[0] = 0.1 * (1.0 / (1.0 + exp(-logits[0])) - al) / n;
        for (int i = 1; i < ORC_CLS_OUT; ++i) g[i] = 0.0;
        if (hit_star[r]) {
            int c, f;
            orc_cls_segment(m_star[r], &c, &f);
            for (int i = 0; i < ORC_CLS_NC; ++i) {
                const double v = logits[1 + i], y = i == c ? 1.0 : 0.0;
                loss += bce_logit(v, y) / ORC_CLS_NC / n_hit;
                g[1 + i] = (1.0 / (1.0 + exp(-v)) - y) / ORC_CLS_NC / n_hit;
            }
            for (int i = 0; i < ORC_CLS_NF; ++i) {
                const double v = logits[1 + ORC_CLS_NC + i], y = i == f ? 1.0 : 0.0;
                loss += bce_logit(v, y) / ORC_CLS_NF / n_hit;
                g[1 + ORC_CLS_NC + i] = (1.0 / (1.0 + exp(-v)) - y) / ORC_CLS_NF / n_hit;
            }
        }
        /* tails: dW = g h^T, db = g, dh = W^T g */
        const double *h16 = hs + (size_t)ORC_CLS_BLOCKS * ORC_CLS_W;
        for (int i = 0; i < ORC_CLS_W; ++i) dh[i] = 0.0;
        for (int s = 0; s < 2; ++s) {
            const int no = s == 0 ? 1 + ORC_CLS_NC : ORC_CLS_NF, g0 = s == 0 ? 0 : 1 + ORC_CLS_NC;
            const size_t off = cls_tail_off() + (s == 0 ? 0 : (size_t)(1 + ORC_CLS_NC) * (ORC_CLS_W + 1));
            for (int o = 0; o < no; ++o) {
                for (int i = 0; i < ORC_CLS_W; ++i) {
                    grad[off + (size_t)o * ORC_CLS_W + i] += g[g0 + o] * h16[i];
                    dh[i] += w[off + (size_t)o * ORC_CLS_W + i] * g[g0 + o];
                }
                grad[off + (size_t)no * ORC_CLS_W + o] += g[g0 + o];
            }
        }
        /* blocks, last to first */
        for (int k = ORC_CLS_BLOCKS - 1; k >= 0; --k) {
            const size_t o1 = cls_block_off(k), o2 = o1 + ORC_CLS_W * ORC_CLS_W + ORC_CLS_W;
            const double *h = hs + (size_t)k * ORC_CLS_W, *u = us + (size_t)k * ORC_CLS_W, *z = zs + (size_t)k * ORC_CLS_W;
            for (int i = 0; i < ORC_CLS_W; ++i) dz[i] = z[i] > 0.0 ? dh[i] : 0.0;
            for (int i = 0; i < ORC_CLS_W; ++i) dt[i] = 0.0;
            for (int o = 0; o < ORC_CLS_W; ++o) {
                for (int i = 0; i < ORC_CLS_W; ++i) {
                    const double ti = dmax(u[i], 0.0);
                    grad[o2 + (size_t)o * ORC_CLS_W + i] += dz[o] * ti;
                    dt[i] += w[o2 + (size_t)o * ORC_CLS_W + i] * dz[o];
                }
                grad[o2 + (size_t)ORC_CLS_W * ORC_CLS_W + o] += dz[o];
            }
            for (int i = 0; i < ORC_CLS_W; ++i) du[i] = u[i] > 0.0 ? dt[i] : 0.0;
            for (int i = 0; i < ORC_CLS_W; ++i) dh[i] = dz[i];       /* the skip connection */
            for (int o = 0; o < ORC_CLS_W; ++o) {
                for (int i = 0; i < ORC_CLS_W; ++i) {
                    grad[o1 + (size_t)o * ORC_CLS_W + i] += du[o] * h[i];
                    dh[i] += w[o1 + (size_t)o * ORC_CLS_W + i] * du[o];
                }
                grad[o1 + (size_t)ORC_CLS_W * ORC_CLS_W + o] += du[o];
            }
        }
        /* head (linear) */
        for (int o = 0; o < ORC_CLS_W; ++o) {
            for (int i = 0; i < ORC_CLS_IN; ++i) grad[(size_t)o * ORC_CLS_IN + i] += dh[o] * xr[i];
            grad[(size_t)ORC_CLS_IN * ORC_CLS_W + o] += dh[o];
        }
    }
    free(hs); free(us); free(zs);
    return loss;
}

/* ------------------------------------------------------------------------------------------ */
/* Depth queries: EXACT (analytic root), MARCH (plain method), MLP (NeDF, Eq. 1-2)              */
/* ------------------------------------------------------------------------------------------ */
static double march_root_sdf(int kind, const double *params, const double ol[3], const double dl[3],
                             double te, double tx, int n, int b, int *hit)
{
    /* Dense scan for the first outside -> inside change of sign of the distance, then bisection. */
    double prev_t = te, x[3];
    for (int c = 0; c < 3; ++c) x[c] = ol[c] + te * dl[c];
    int prev_in = orc_sdf(kind, params, x) <= 0.0;
    for (int k = 1; k <= n; ++k) {
        double t = te + (tx - te) * k / n;
        for (int c = 0; c < 3; ++c) x[c] = ol[c] + t * dl[c];
        int in = orc_sdf(kind, params, x) <= 0.0;
        if (in && !prev_in) {
            double lo = prev_t, hi = t;
            for (int it = 0; it < b; ++it) {
                double mid = 0.5 * (lo + hi);
                for (int c = 0; c < 3; ++c) x[c] = ol[c] + mid * dl[c];
                if (orc_sdf(kind, params, x) <= 0.0) hi = mid; else lo = mid;
            }
            *hit = 1;
            return 0.5 * (lo + hi);
        }
        prev_in = in;
        prev_t = t;
    }
    *hit = 0;
    return INFINITY;
}

double orc_exact_depth(int kind, const double *p, const double ol[3], const double dl[3],
                       double te, double tx, int *hit)
{
    *hit = 0;
    if (kind == ORC_SPHERE) {
        double b = dot3(ol, dl), c = dot3(ol, ol) - p[0] * p[0], disc = b * b - c;
        if (disc < 0.0) return INFINITY;
        double t0 = -b - sqrt(disc);
        if (t0 >= te && t0 <= tx) { *hit = 1; return t0; }
        return INFINITY;
    }
    if (kind == ORC_BOX) { /* slab method */
        double tn = -INFINITY, tf = INFINITY;
        for (int c = 0; c < 3; ++c) {
            if (dl[c] == 0.0) {
                if (fabs(ol[c]) > p[c]) return INFINITY;
                continue;
            }
            double t1 = (-p[c] - ol[c]) / dl[c], t2 = (p[c] - ol[c]) / dl[c];
            tn = dmax(tn, dmin(t1, t2));
            tf = dmin(tf, dmax(t1, t2));
        }
        if (tn <= tf && tn >= te && tn <= tx) { *hit = 1; return tn; }
        return INFINITY;
    }
    /* No closed form in use: converge a fine scan of the distance's sign change. */
    return march_root_sdf(kind, p, ol, dl, te, tx, 20000, 80, hit);
}

/* Plain method (our reading of the label depth): N uniform steps over [te, tx], the first step
 * whose density reaches sigma_max/2 after one below it, then B bisection steps; midpoint. */
/* Depth-decision diagnostics of one query (diagnostic only; the depth itself does not use them).
 * Every inside/outside test at a point x = ol + t dl has a margin, |sdf(x)| (the distance the
 * point may move before the test changes, the SDFs being distance bounds) less the shift `u`
 * another implementation's inputs may carry, relative to the coordinate magnitude |ol| + |t| + rb
 * that bounds its rounding error; and a consequence, how far the depth can move if the test goes
 * the other way: half the bracket for a bisection step, unbounded for the plain method's samples
 * and the refinement window's ends (a crossing found elsewhere or not at all, an outlier). */
#define ORC_DEC_CAP 1e-4      /* tests with a larger margin are never knife edges: not recorded */
#define ORC_DEC_MAX 32
typedef struct {
    int count;                  /* tests taken so far (a test's index) */
    int flip;                   /* index of a test to take the other way (-1: none) */
    int n;                      /* recorded tests with a margin below ORC_DEC_CAP */
    double m[ORC_DEC_MAX], c[ORC_DEC_MAX];
    int idx[ORC_DEC_MAX];
} dec_diag;

static void dec_init(dec_diag *g, int flip) { g->count = 0; g->flip = flip; g->n = 0; }

/* One inside/outside test at x = ol + t dl (the half-density level, reading 9) with margin
 * bookkeeping; taken the other way when it is the test to flip. */
static int decide(dec_diag *g, const orc_scene *sc, int type, const double ol[3], double t, const double x[3],
                  double u, double consequence)
{
    int in = inside_solid(sc, type, x);
    if (!g) return in;
    const orc_type *ty = &sc->types[type];
    double mg = dmax(fabs(orc_sdf(ty->kind, ty->params, x)) - u, 0.0) / (len3(ol) + fabs(t) + ty->rb);
    if (mg < ORC_DEC_CAP) {
        int slot = g->n;
        if (g->n == ORC_DEC_MAX) {              /* full: replace the largest margin if larger */
            slot = 0;
            for (int i = 1; i < ORC_DEC_MAX; ++i) if (g->m[i] > g->m[slot]) slot = i;
            if (g->m[slot] <= mg) slot = -1;
        } else {
            ++g->n;
        }
        if (slot >= 0) { g->m[slot] = mg; g->c[slot] = consequence; g->idx[slot] = g->count; }
    }
    if (g->count == g->flip) in = !in;
    ++g->count;
    return in;
}

/* The smallest margin among the recorded tests whose consequence reaches `need` (local length). */
static double dec_margin(const dec_diag *g, double need)
{
    double r = INFINITY;
    for (int i = 0; i < g->n; ++i)
        if (g->c[i] >= need) r = dmin(r, g->m[i]);
    return r;
}

/* The two most critical tests of a pixel, each named by where it ran: stage 1 = the Step-1 query
 * of instance `inst` (stage 0: none); idx = its index in that query. */
typedef struct { double m; int stage, light, inst, idx; } crit_test;

static void crit_feed(crit_test cr[2], const dec_diag *g, double need, int stage, int light, int inst)
{
    for (int i = 0; i < g->n; ++i) {
        if (!(g->c[i] >= need)) continue;
        crit_test t = {g->m[i], stage, light, inst, g->idx[i]};
        if (t.m < cr[0].m) { cr[1] = cr[0]; cr[0] = t; }
        else if (t.m < cr[1].m) cr[1] = t;
    }
}

static double march_core(const orc_scene *sc, int type, const double ol[3], const double dl[3], double te,
                         double tx, int n, int b, int *hit, dec_diag *dg)
{
    double x[3], prev_t = te;
    for (int c = 0; c < 3; ++c) x[c] = ol[c] + te * dl[c];
    int prev_in = decide(dg, sc, type, ol, te, x, 0.0, INFINITY);
    for (int k = 1; k <= n; ++k) {
        double t = te + (tx - te) * k / n;
        for (int c = 0; c < 3; ++c) x[c] = ol[c] + t * dl[c];
        int in = decide(dg, sc, type, ol, t, x, 0.0, INFINITY);
        if (in && !prev_in) {
            double lo = prev_t, hi = t;
            for (int it = 0; it < b; ++it) {
                double mid = 0.5 * (lo + hi);
                for (int c = 0; c < 3; ++c) x[c] = ol[c] + mid * dl[c];
                if (decide(dg, sc, type, ol, mid, x, 0.0, 0.5 * (hi - lo))) hi = mid; else lo = mid;
            }
            *hit = 1;
            return 0.5 * (lo + hi);
        }
        prev_in = in;
        prev_t = t;
    }
    *hit = 0;
    return INFINITY;
}

double orc_march_depth(const orc_scene *sc, int type, const double ol[3], const double dl[3],
                       double te, double tx, int n, int b, int *hit)
{
    return march_core(sc, type, ol, dl, te, tx, n, b, hit, NULL);
}

/* Network-rounding spread of a regression NeDF row in the BF16 / E4M3 modes: the largest change of
 * (m, a) when one of its ORC_FLIP_CAND values nearest to a rounding boundary (relative margin below
 * the format's limit, i.e. within reach of another implementation's sums) rounds the other way. */
#define ORC_FLIP_CAND 16
/* BF16: FP32 sums plus a bias carried to ~16 significant bits (relative 2^-17 of |b|); E4M3: the
 * accumulation of E4M3 products, coarser than FP32 (flips measured at relative margins to ~1e-4) */
#define ORC_FLIP_MARGIN_BF16 2e-5
#define ORC_FLIP_MARGIN_FP8 2e-5
static void nedf_spread(const orc_type *t, const int *dims, int nl, const double *feat, const double y[2],
                        int quant, double spread[2])
{
    spread[0] = spread[1] = 0.0;
    if (quant == ORC_QUANT_NONE || t->nedf_arch == ORC_ARCH_CLASSIFIER) return;
    const double lim = quant == ORC_QUANT_FP8 ? ORC_FLIP_MARGIN_FP8 : ORC_FLIP_MARGIN_BF16;
    int ci[ORC_FLIP_CAND];
    double cm[ORC_FLIP_CAND], yf[2];
    mlp_core(t->nedf_w, nl, dims, feat, yf, quant, NULL, -1, ORC_FLIP_CAND, ci, cm);
    for (int c = 0; c < ORC_FLIP_CAND; ++c) {
        if (ci[c] < 0 || !(cm[c] < lim)) break;
        mlp_core(t->nedf_w, nl, dims, feat, yf, quant, NULL, ci[c], 0, NULL, NULL);
        spread[0] = dmax(spread[0], fabs(yf[0] - y[0]));
        spread[1] = dmax(spread[1], fabs(yf[1] - y[1]));
    }
}

/* One (ray, instance) query of Step 1 / Step 3 with its knife-edge diagnostics:
 *   *margin   distance of the query's discrete decisions from their thresholds (cull
 *             discriminant, bound exit, hit logit, D > 0, fallback confidence, the depth check's
 *             window ends), each reduced by the network-rounding spread it can move by;
 *   *dg       the depth-decision diagnostics (dec_diag) of the plain method's tests and of the
 *             refinement (none when the depth comes from the network alone);
 *   *dspread  the local depth shift a single network-rounding flip can cause (rb times the
 *             spread of m; 0 for depths from the plain method). */
static int query_ex(const orc_scene *sc, const orc_opts *op, int inst, const double o[3], const double d[3],
                    double out6[6], double *margin, dec_diag *dg, int flip, double *dspread)
{
    const orc_type *t = &sc->types[sc->inst_type[inst]];
    const int type = sc->inst_type[inst];
    double ol[3], dl[3], bd[4], feat[ORC_CLS_IN];
    orc_to_local(sc, inst, o, d, ol, dl);
    int kept = t->nedf_arch == ORC_ARCH_CLASSIFIER ? orc_cls_features(ol, dl, t->rb, feat, bd)
                                                   : orc_nedf_features(ol, dl, t->rb, feat, bd);
    double mg = fabs(bd[3]) / (t->rb * t->rb), dsp = 0.0;
    dec_init(dg, flip);
    if (kept) mg = dmin(mg, fabs(bd[1]) / t->rb);
    out6[0] = INFINITY; out6[1] = out6[2] = 0.0;
    out6[3] = bd[0]; out6[4] = bd[1]; out6[5] = bd[2];
    if (!kept) { *margin = mg; *dspread = dsp; return 0; }
    int hit = 0;
    double Dl = INFINITY;
    if (op->depth_mode == ORC_DEPTH_EXACT) {
        Dl = orc_exact_depth(t->kind, t->params, ol, dl, bd[0], bd[1], &hit);
    } else if (op->depth_mode == ORC_DEPTH_MARCH) {
        Dl = march_core(sc, type, ol, dl, bd[0], bd[1], op->march_n, op->march_b, &hit, dg);
    } else {
        /* Eq. 1: F_Phi(r) -> (mu, alpha); mu = l * m with l = rb (reading: the mu range [-l, l]
         * is the bound sphere's).  Eq. 2: D = |o - p_perp| - mu with the signed t_perp. */
        double y[2], spread[2] = {0.0, 0.0};
        if (t->nedf_arch == ORC_ARCH_CLASSIFIER) {
            /* Eq. 3-4: the two-level classifier's argmax bins give m = mu / l */
            double logits[ORC_CLS_OUT];
            int c, f;
            orc_cls_forward(op->quant == ORC_QUANT_NONE ? t->nedf_w : t->nedf_wq, feat, logits, op->quant);
            mg = dmin(mg, orc_cls_decode(logits, &y[0], &y[1], &c, &f));
        } else {
            int dims[64], nl = nedf_dims(t, dims);
            orc_mlp(t->nedf_w, nl, dims, feat, y, op->quant);
            nedf_spread(t, dims, nl, feat, y, op->quant, spread);
        }
        out6[1] = y[0];
        out6[2] = y[1];
        Dl = bd[2] - t->rb * y[0];
        dsp = t->rb * spread[0];
        hit = (y[1] > 0.0) && (Dl > 0.0);
        mg = dmin(mg, dmin(fabs(y[1]) - spread[1], (fabs(Dl) - dsp) / t->rb));
        /* Low-confidence pairs are re-answered by the plain method. */
        int march = 0;
        if (op->fallback_conf > 0.0) {
            double pr = 1.0 / (1.0 + exp(-y[1]));
            double conf = dmax(pr, 1.0 - pr);
            /* d conf / d a is at most 1/4 */
            mg = dmin(mg, fabs(conf - op->fallback_conf) - 0.25 * spread[1]);
            march = conf < op->fallback_conf;
        }
        /* Check of a confident NeDF miss (reading 30): the density at miss_check midpoints of the
         * bound chord; reaching the half level at one makes the miss wrong, re-answered by the
         * plain method. */
        if (!march && !hit && op->miss_check > 0) {
            double x[3];
            for (int j = 0; j < op->miss_check && !march; ++j) {
                const double tj = bd[0] + (j + 0.5) * (bd[1] - bd[0]) / op->miss_check;
                for (int c = 0; c < 3; ++c) x[c] = ol[c] + tj * dl[c];
                march = decide(dg, sc, type, ol, tj, x, 0.0, INFINITY);
            }
        }
        /* Depth check of a NeDF hit (Section "Deferred Shading": the density at the predicted
         * depth tells whether it reached the surface): if the half-density level is crossed
         * inside [D - h, D + h], bisect it; otherwise the hit is an outlier, re-answered by the
         * plain method when outlier_resample is set. */
        if (!march && hit && op->refine_steps > 0) {
            double lo = Dl - sc->shade_half, hi = Dl + sc->shade_half, x[3];
            for (int c = 0; c < 3; ++c) x[c] = ol[c] + lo * dl[c];
            int in_lo = decide(dg, sc, type, ol, lo, x, dsp, INFINITY);
            mg = dmin(mg, fabs(orc_sdf(t->kind, t->params, x)) - dsp);
            for (int c = 0; c < 3; ++c) x[c] = ol[c] + hi * dl[c];
            int in_hi = decide(dg, sc, type, ol, hi, x, dsp, INFINITY);
            mg = dmin(mg, fabs(orc_sdf(t->kind, t->params, x)) - dsp);
            if (!in_lo && in_hi) {
                for (int it = 0; it < op->refine_steps; ++it) {
                    double mid = 0.5 * (lo + hi);
                    for (int c = 0; c < 3; ++c) x[c] = ol[c] + mid * dl[c];
                    if (decide(dg, sc, type, ol, mid, x, dsp, 0.5 * (hi - lo))) hi = mid; else lo = mid;
                }
                Dl = 0.5 * (lo + hi);
                hit = Dl > 0.0;
                mg = dmin(mg, (fabs(Dl) - dsp) / t->rb);
            } else if (op->outlier_resample) {
                march = 1;
            }
        }
        if (march) {
            Dl = march_core(sc, type, ol, dl, bd[0], bd[1], op->march_n, op->march_b, &hit, dg);
            dsp = 0.0;
        }
    }
    out6[0] = Dl;
    *margin = mg;
    *dspread = dsp;
    return hit;
}

int orc_query(const orc_scene *sc, const orc_opts *op, int inst, const double o[3], const double d[3],
              double out6[6], double *margin)
{
    double dsp;
    dec_diag dg;
    return query_ex(sc, op, inst, o, d, out6, margin, &dg, -1, &dsp);
}

int orc_query_diag(const orc_scene *sc, const orc_opts *op, int inst, const double o[3], const double d[3],
                   double out6[6], double diag[3], double need)
{
    dec_diag dg;
    int hit = query_ex(sc, op, inst, o, d, out6, &diag[0], &dg, -1, &diag[2]);
    diag[1] = dec_margin(&dg, need);
    return hit;
}

/* ------------------------------------------------------------------------------------------ */
/* Step 2: deferred shading (Eq. 8 with n samples in a window around the stored depth)          */
/* ------------------------------------------------------------------------------------------ */
void orc_composite_samples(int n, const double *sigma, const double *rgb, double world_delta, double rgba[4])
{
    double T = 1.0;
    rgba[0] = rgba[1] = rgba[2] = rgba[3] = 0.0;
    for (int j = 0; j < n; ++j) {
        double alpha = 1.0 - exp(-sigma[j] * world_delta);
        for (int c = 0; c < 3; ++c) rgba[c] += T * alpha * rgb[3 * j + c];
        rgba[3] += T * alpha;
        T *= 1.0 - alpha;
    }
}

static void sample_colour(const orc_type *t, const double x[3], const double dl[3], int quant, double rgb[3])
{
    if (t->nerf_hidden == 0) {
        for (int c = 0; c < 3; ++c) rgb[c] = t->albedo[c];
        return;
    }
    double feat[90], y[3];
    int dims[64], nl = nerf_dims(t, dims);
    orc_posenc(x, 3, 10, feat);
    orc_posenc(dl, 3, 4, feat + 63);
    orc_mlp(t->nerf_w, nl, dims, feat, y, quant);
    for (int c = 0; c < 3; ++c) rgb[c] = 1.0 / (1.0 + exp(-y[c]));
}

/* Step 2 for one pixel; returns the largest sample density (the outlier test of "rs") */
static double shade_pixel(const orc_scene *sc, const orc_opts *op, const double o[3], const double d[3],
                          int inst, double depth, double rgba[4])
{
    const orc_type *t = &sc->types[sc->inst_type[inst]];
    double ol[3], dl[3], s = sc->inst_s[inst];
    orc_to_local(sc, inst, o, d, ol, dl);
    double Dl = depth / s, h = sc->shade_half;
    int n = sc->n_shade;
    double delta = 2.0 * h / n;
    double *sig = (double *)malloc(sizeof(double) * n), *rgb = (double *)malloc(sizeof(double) * 3 * n);
    for (int j = 0; j < n; ++j) {
        double tj = Dl - h + (j + 0.5) * delta, x[3];
        for (int c = 0; c < 3; ++c) x[c] = ol[c] + tj * dl[c];
        sig[j] = orc_density(sc, sc->inst_type[inst], x);
        sample_colour(t, x, dl, op->quant, rgb + 3 * j);
    }
    orc_composite_samples(n, sig, rgb, s * delta, rgba);
    double smax = 0.0;
    for (int j = 0; j < n; ++j) smax = dmax(smax, sig[j]);
    free(sig);
    free(rgb);
    return smax;
}

/* The plain method's colour of one pixel (defined with the volume renderer below). */
typedef struct { double te_world; int inst; } vr_pair;
static void vr_pixel(const orc_scene *sc, const orc_opts *op, int ns, int64_t p, vr_pair *pairs, double rgba[4],
                     double *vmargin);

/* ------------------------------------------------------------------------------------------ */
/* Algorithm 1 (Steps 1-2) and Algorithm 2 (Step 3) for one pixel                               */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    const orc_scene *sc;
    const orc_opts *op;
    const int64_t *px;
    int64_t begin, end;
    double *depth, *gap, *pmargin, *rgba, *shadow, *smargin, *out, *shade_smax, *dmargin;
    uint32_t *id;
    double *alt;                 /* per pixel: depth, id (as double), rgba[4], shadow, out[4] */
} render_job;

#define ORC_ALT_MARGIN 1e-6      /* pixels whose most critical depth test is closer get an alternative */
/* The depth tolerance of the comparisons (1e-3 relative, 2e-3 absolute: the FP32 contract of the
 * render path): a depth test whose consequence stays below it cannot decide a depth comparison. */
#define ORC_DEPTH_TOL_ABS 2e-3
#define ORC_DEPTH_TOL_REL 1e-3

typedef struct {
    double depth, gap, pm, sm, smax, rgba[4], S;
    uint32_t id;
} pixel_result;

/* Steps 2 and 3 of pixel p (camera ray o, d) given its winning instance `inst` and world depth:
 * the shading of Eq. 8 over the sample window (or the plain method's colour for an outlier with
 * resampling), then the shadow rays of Algorithm 2.  rgba, *S (the shadow factor), *sm (the shadow
 * tests' margin, 0 where a depth test of a shadow query could move its depth across the test) and
 * *smax (the largest sample density) are written. */
static void steps23(const orc_scene *sc, const orc_opts *op, int64_t p, const double o[3], const double d[3], int inst,
                    double depth, double rgba[4], double *S_out, double *sm_out, double *smax_out)
{
    double q[6], mg, dsp, S = 1.0, sm = INFINITY, smax = NAN;
    dec_diag dg;
    {
        /* STEP 2: shade with the winning model's radiance field only. */
        smax = shade_pixel(sc, op, o, d, inst, depth, rgba);
        /* Outlier resampling: an extremely small density says the depth missed the surface; the
         * pixel's colour then comes from the primary volume rendering of every model. */
        if (op->shade_resample > 0 && smax < op->shade_sigma_min) {
            vr_pair *buf = (vr_pair *)malloc(sizeof(vr_pair) * (sc->n_inst > 0 ? sc->n_inst : 1));
            vr_pixel(sc, op, op->shade_resample, p, buf, rgba, NULL);
            free(buf);
        }
        /* STEP 3: x on the surface, shadow ray from each light towards x; an occluder hit
         * closer to the light than x by more than eps darkens by beta; lights averaged. */
        double x[3];
        for (int c = 0; c < 3; ++c) x[c] = o[c] + depth * d[c];
        double acc = 0.0;
        for (int l = 0; l < sc->n_lights; ++l) {
            const double *L = sc->lights + 3 * l;
            double Lp[3];
            if (sc->light_parallel && sc->light_parallel[l]) {
                /* A parallel light reaches x from infinity along its direction w: the shadow ray
                 * starts on that line beyond every object's bound (any such start gives the same
                 * answers: the same entry points and directions, the same order along the ray). */
                double w[3] = {L[0], L[1], L[2]}, wl = len3(w), far = 1.0 + len3(x);
                for (int m = 0; m < sc->n_inst; ++m) {
                    const double *Tm = sc->inst_T + 3 * m;
                    far = dmax(far, 2.0 * (len3(Tm) + sc->inst_s[m] * sc->types[sc->inst_type[m]].rb + len3(x)));
                }
                for (int c = 0; c < 3; ++c) Lp[c] = x[c] - far * w[c] / wl;
                L = Lp;
            }
            double v[3] = {x[0] - L[0], x[1] - L[1], x[2] - L[2]};
            double ell = len3(v), dir[3] = {v[0] / ell, v[1] / ell, v[2] / ell};
            int occluded = 0;
            for (int m = 0; m < sc->n_inst; ++m) {
                int hit = query_ex(sc, op, m, L, dir, q, &mg, &dg, -1, &dsp);
                double s = sc->inst_s[m];
                if (!(q[3] <= q[4]) || q[4] < 0.0) { sm = dmin(sm, mg); continue; } /* culled */
                /* Reading: only bounds the shadow segment enters before x can occlude x. */
                sm = dmin(sm, fabs(q[3] * s - ell));
                if (!(q[3] * s < ell)) continue;
                sm = dmin(sm, mg);
                /* a depth test of this query that could go the other way (margin below
                 * ORC_ALT_MARGIN) and move its depth across the shadow test makes the test a knife
                 * edge */
                if (!hit) {
                    if (dec_margin(&dg, INFINITY) < ORC_ALT_MARGIN) sm = 0.0;
                    continue;
                }
                double Dk = s * q[0];
                sm = dmin(sm, fabs(Dk + sc->eps - ell) - s * dsp);
                if (dec_margin(&dg, fabs(Dk + sc->eps - ell) / s) < ORC_ALT_MARGIN) sm = 0.0;
                if (Dk + sc->eps < ell) occluded = 1;
            }
            acc += occluded ? sc->beta : 1.0;
        }
        S = acc / sc->n_lights;
    }
    *S_out = S;
    *sm_out = sm;
    *smax_out = smax;
}

/* Steps 1-3 for pixel p.  `fl` names one depth test to take the other way (stage 0: none);
 * cr[2] receives the pixel's two most critical depth tests (see render_one). */
static void render_pixel(const orc_scene *sc, const orc_opts *op, int64_t p, const crit_test *fl,
                         pixel_result *r, crit_test cr[2])
{
    int i = (int)(p % sc->W), j = (int)(p / sc->W);
    double o[3], d[3], q[6], mg, dsp, best = INFINITY, second = INFINITY, pm = INFINITY;
    double u_best = 0.0, u_second = 0.0;
    uint32_t bid = 0xFFFFFFFFu;
    cr[0].m = cr[1].m = INFINITY;
    cr[0].stage = cr[1].stage = 0;
    orc_camera_ray(sc, i, j, o, d);
    /* STEP 1: clear to infinity; visit models in id order; strict '<' keeps the lowest id on ties. */
    const int ni = sc->n_inst > 0 ? sc->n_inst : 1;
    double *Dq = (double *)malloc(sizeof(double) * ni);
    dec_diag *dq = (dec_diag *)malloc(sizeof(dec_diag) * ni);
    for (int m = 0; m < sc->n_inst; ++m) {
        int flip = (fl->stage == 1 && fl->inst == m) ? fl->idx : -1;
        int hit = query_ex(sc, op, m, o, d, q, &mg, &dq[m], flip, &dsp);
        pm = dmin(pm, mg);
        Dq[m] = hit ? sc->inst_s[m] * q[0] : INFINITY;
        if (!hit) { crit_feed(cr, &dq[m], INFINITY, 1, 0, m); continue; }   /* could it become a hit? */
        double D = Dq[m], u = sc->inst_s[m] * dsp;
        if (D < best) { second = best; u_second = u_best; best = D; u_best = u; bid = (uint32_t)m; }
        else if (D < second) { second = D; u_second = u; }
    }
    /* Depth tests that can change this pixel's Step-1 result: the winner's whose consequence
     * reaches the depth tolerance (ORC_DEPTH_TOL_*: Steps 2-3 are answered for a given depth by
     * orc_steps23), and those of each other hit whose consequence reaches the winner. */
    for (int m = 0; m < sc->n_inst; ++m) {
        if (!isfinite(Dq[m])) continue;
        const double need = (uint32_t)m == bid ? dmax(ORC_DEPTH_TOL_ABS, ORC_DEPTH_TOL_REL * best) : Dq[m] - best;
        crit_feed(cr, &dq[m], need / sc->inst_s[m], 1, 0, m);
    }
    free(Dq);
    free(dq);
    double rgba[4] = {0, 0, 0, 0}, S = 1.0, sm = INFINITY, smax = NAN;
    if (bid != 0xFFFFFFFFu) steps23(sc, op, p, o, d, (int)bid, best, rgba, &S, &sm, &smax);
    r->depth = best;
    r->id = bid;
    /* the gap less the depth shift single network-rounding flips can cause on either side */
    r->gap = (bid != 0xFFFFFFFFu) ? second - best - u_best - u_second : INFINITY;
    r->pm = pm;
    r->sm = sm;
    r->smax = smax;
    for (int c = 0; c < 4; ++c) r->rgba[c] = rgba[c];
    r->S = S;
}

/* Pixel k of the job.  dmargin is the margin of its most critical depth test.  When that is below
 * ORC_ALT_MARGIN the pixel is rendered a second time with that one test taken the other way (what
 * an implementation whose coordinates differ by rounding may do) into `alt`, and dmargin becomes
 * the margin of the second most critical test: the alternative covers the first. */
static void render_one(const render_job *jb, int64_t k)
{
    const orc_scene *sc = jb->sc;
    const orc_opts *op = jb->op;
    const crit_test none = {INFINITY, 0, 0, 0, -1};
    crit_test cr[2], cr2[2];
    pixel_result r, ra;
    render_pixel(sc, op, jb->px[k], &none, &r, cr);
    double dm = cr[0].m;
    int has_alt = jb->alt && cr[0].m < ORC_ALT_MARGIN;
    if (has_alt) {
        render_pixel(sc, op, jb->px[k], &cr[0], &ra, cr2);
        dm = cr[1].m;
    }
    jb->depth[k] = r.depth;
    jb->id[k] = r.id;
    if (jb->gap) jb->gap[k] = r.gap;
    if (jb->pmargin) jb->pmargin[k] = r.pm;
    if (jb->dmargin) jb->dmargin[k] = dm;
    if (jb->rgba) for (int c = 0; c < 4; ++c) jb->rgba[4 * k + c] = r.rgba[c];
    if (jb->shadow) jb->shadow[k] = r.S;
    if (jb->smargin) jb->smargin[k] = r.sm;
    if (jb->shade_smax) jb->shade_smax[k] = r.smax;
    if (jb->out) {
        for (int c = 0; c < 3; ++c) jb->out[4 * k + c] = r.rgba[c] * r.S;
        jb->out[4 * k + 3] = r.rgba[3];
    }
    if (jb->alt) {
        double *a = jb->alt + 12 * k;
        if (has_alt) {
            a[0] = ra.depth;
            a[1] = ra.id == 0xFFFFFFFFu ? -1.0 : (double)ra.id;
            for (int c = 0; c < 4; ++c) a[2 + c] = ra.rgba[c];
            a[6] = ra.S;
            for (int c = 0; c < 3; ++c) a[7 + c] = ra.rgba[c] * ra.S;
            a[10] = ra.rgba[3];
            a[11] = 1.0;
        } else {
            for (int c = 0; c < 12; ++c) a[c] = NAN;
            a[11] = 0.0;
        }
    }
}

static void *render_worker(void *arg)
{
    const render_job *jb = (const render_job *)arg;
    for (int64_t k = jb->begin; k < jb->end; ++k) render_one(jb, k);
    return NULL;
}

int orc_render(const orc_scene *sc, const orc_opts *op, int64_t n_px, const int64_t *px, double *depth,
               uint32_t *id, double *gap, double *pmargin, double *rgba, double *shadow, double *smargin,
               double *out, double *shade_smax, double *dmargin, double *alt)
{
    int nt = op->n_threads > 1 ? op->n_threads : 1;
    if (nt > 256) nt = 256;
    render_job jobs[256];
    pthread_t th[256];
    for (int t = 0; t < nt; ++t) {
        render_job jb = {sc, op, px, n_px * t / nt, n_px * (t + 1) / nt, depth, gap, pmargin, rgba,
                         shadow, smargin, out, shade_smax, dmargin, id, alt};
        jobs[t] = jb;
    }
    if (nt == 1) { render_worker(&jobs[0]); return 0; }
    for (int t = 0; t < nt; ++t) pthread_create(&th[t], NULL, render_worker, &jobs[t]);
    for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
    return 0;
}

/* Steps 2-3 alone for pixels whose winner and world depth are given (id 0xFFFFFFFF: no hit). */
typedef struct {
    const orc_scene *sc;
    const orc_opts *op;
    const int64_t *px;
    const uint32_t *id;
    const double *depth;
    int64_t begin, end;
    double *rgba, *shadow, *smargin, *out;
} s23_job;

static void *s23_worker(void *arg)
{
    const s23_job *jb = (const s23_job *)arg;
    for (int64_t k = jb->begin; k < jb->end; ++k) {
        double rgba[4] = {0, 0, 0, 0}, S = 1.0, sm = INFINITY, smax = NAN;
        if (jb->id[k] != 0xFFFFFFFFu && (int64_t)jb->id[k] < jb->sc->n_inst) {
            double o[3], d[3];
            const int64_t p = jb->px[k];
            orc_camera_ray(jb->sc, (int)(p % jb->sc->W), (int)(p / jb->sc->W), o, d);
            steps23(jb->sc, jb->op, p, o, d, (int)jb->id[k], jb->depth[k], rgba, &S, &sm, &smax);
        }
        for (int c = 0; c < 4; ++c) jb->rgba[4 * k + c] = rgba[c];
        jb->shadow[k] = S;
        jb->smargin[k] = sm;
        for (int c = 0; c < 3; ++c) jb->out[4 * k + c] = rgba[c] * S;
        jb->out[4 * k + 3] = rgba[3];
    }
    return NULL;
}

int orc_steps23(const orc_scene *sc, const orc_opts *op, int64_t n_px, const int64_t *px, const uint32_t *id,
                const double *depth, double *rgba, double *shadow, double *smargin, double *out)
{
    int nt = op->n_threads > 1 ? op->n_threads : 1;
    if (nt > 256) nt = 256;
    s23_job jobs[256];
    pthread_t th[256];
    for (int t = 0; t < nt; ++t) {
        s23_job jb = {sc, op, px, id, depth, n_px * t / nt, n_px * (t + 1) / nt, rgba, shadow, smargin, out};
        jobs[t] = jb;
    }
    if (nt == 1) { s23_worker(&jobs[0]); return 0; }
    for (int t = 0; t < nt; ++t) pthread_create(&th[t], NULL, s23_worker, &jobs[t]);
    for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Plain method colour: every NeRF volume-rendered front to back (ordered by entry distance)    */
/* ------------------------------------------------------------------------------------------ */
static int cmp_pair(const void *a, const void *b)
{
    const vr_pair *x = (const vr_pair *)a, *y = (const vr_pair *)b;
    if (x->te_world < y->te_world) return -1;
    if (x->te_world > y->te_world) return 1;
    return x->inst - y->inst;
}

typedef struct {
    const orc_scene *sc; const orc_opts *op; int ns; const int64_t *px; int64_t begin, end; double *rgba, *vmargin;
} vr_job;

/* Pixel p: its (ray, model) pairs that meet the bounds, front to back by (entry distance, id),
 * each volume rendered with ns midpoint samples over its chord.  *vmargin (may be NULL) receives the
 * distance of its discrete decisions from their thresholds: each bound's cull discriminant over
 * rb^2 and the entry-distance differences that order the pairs (diagnostic only). */
static void vr_pixel(const orc_scene *sc, const orc_opts *op, int ns, int64_t p, vr_pair *pairs, double rgba[4],
                     double *vmargin)
{
    double o[3], d[3], ol[3], dl[3], bd[4], vm = INFINITY;
    orc_camera_ray(sc, (int)(p % sc->W), (int)(p / sc->W), o, d);
    int np = 0;
    for (int m = 0; m < sc->n_inst; ++m) {
        orc_to_local(sc, m, o, d, ol, dl);
        double rb = sc->types[sc->inst_type[m]].rb;
        int kept = orc_bound(ol, dl, rb, bd);
        vm = dmin(vm, fabs(bd[3]) / (rb * rb));
        if (!kept) continue;
        pairs[np].te_world = bd[0] * sc->inst_s[m];
        pairs[np].inst = m;
        ++np;
    }
    qsort(pairs, np, sizeof(vr_pair), cmp_pair);
    for (int q = 1; q < np; ++q) vm = dmin(vm, pairs[q].te_world - pairs[q - 1].te_world);
    double T = 1.0, C[3] = {0, 0, 0};
    for (int q = 0; q < np; ++q) {
        int m = pairs[q].inst;
        const orc_type *t = &sc->types[sc->inst_type[m]];
        double s = sc->inst_s[m];
        orc_to_local(sc, m, o, d, ol, dl);
        orc_bound(ol, dl, t->rb, bd);
        double dt = (bd[1] - bd[0]) / ns;
        for (int j = 0; j < ns; ++j) {
            double tj = bd[0] + (j + 0.5) * dt, x[3], rgb[3];
            for (int c = 0; c < 3; ++c) x[c] = ol[c] + tj * dl[c];
            double alpha = 1.0 - exp(-orc_density(sc, sc->inst_type[m], x) * s * dt);
            sample_colour(t, x, dl, op->quant, rgb);
            for (int c = 0; c < 3; ++c) C[c] += T * alpha * rgb[c];
            T *= 1.0 - alpha;
        }
    }
    for (int c = 0; c < 3; ++c) rgba[c] = C[c];
    rgba[3] = 1.0 - T;
    if (vmargin) *vmargin = vm;
}

static void *vr_worker(void *arg)
{
    const vr_job *jb = (const vr_job *)arg;
    const orc_scene *sc = jb->sc;
    vr_pair *pairs = (vr_pair *)malloc(sizeof(vr_pair) * (sc->n_inst > 0 ? sc->n_inst : 1));
    for (int64_t k = jb->begin; k < jb->end; ++k)
        vr_pixel(sc, jb->op, jb->ns, jb->px[k], pairs, jb->rgba + 4 * k, jb->vmargin ? jb->vmargin + k : NULL);
    free(pairs);
    return NULL;
}

int orc_volume_render(const orc_scene *sc, const orc_opts *op, int n_samples, int64_t n_px,
                      const int64_t *px, double *rgba, double *vmargin)
{
    int nt = op->n_threads > 1 ? op->n_threads : 1;
    if (nt > 256) nt = 256;
    vr_job jobs[256];
    pthread_t th[256];
    for (int t = 0; t < nt; ++t) {
        vr_job jb = {sc, op, n_samples, px, n_px * t / nt, n_px * (t + 1) / nt, rgba, vmargin};
        jobs[t] = jb;
    }
    if (nt == 1) { vr_worker(&jobs[0]); return 0; }
    for (int t = 0; t < nt; ++t) pthread_create(&th[t], NULL, vr_worker, &jobs[t]);
    for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Learned part: ray sampler, ray-march labels, loss and hand-derived gradient, Adam            */
/* ------------------------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea & Flood 2014) in counter form: output `index` of the stream `seed`. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t index)
{
    uint64_t z = seed + (index + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double u24(uint64_t seed, uint64_t index)
{
    return (double)(orc_splitmix64(seed, index) >> 40) * (1.0 / 16777216.0);
}

/* Ray r: entry point uniform on the bound sphere, direction cosine-weighted about the inward
 * normal.  Draws 4r .. 4r+3.  The tangent frame is Duff et al. (JCGT 2017). */
void orc_train_rays(double rb, uint64_t seed, int64_t first, int n, double *o, double *d)
{
    for (int k = 0; k < n; ++k) {
        uint64_t r = (uint64_t)(first + k);
        double u0 = u24(seed, 4 * r), u1 = u24(seed, 4 * r + 1), u2 = u24(seed, 4 * r + 2), u3 = u24(seed, 4 * r + 3);
        double z = 1.0 - 2.0 * u0, phi = 2.0 * PI * u1, rho = sqrt(dmax(0.0, 1.0 - z * z));
        double nrm[3] = {rho * cos(phi), rho * sin(phi), z};
        double w[3] = {-nrm[0], -nrm[1], -nrm[2]};
        double sg = w[2] >= 0.0 ? 1.0 : -1.0;
        double a = -1.0 / (sg + w[2]), b = w[0] * w[1] * a;
        double b1[3] = {1.0 + sg * w[0] * w[0] * a, sg * b, -sg * w[0]};
        double b2[3] = {b, sg + w[1] * w[1] * a, -w[1]};
        double rr = sqrt(u2), th = 2.0 * PI * u3;
        double lx = rr * cos(th), ly = rr * sin(th), lz = sqrt(dmax(0.0, 1.0 - u2));
        for (int c = 0; c < 3; ++c) {
            o[3 * k + c] = rb * nrm[c];
            d[3 * k + c] = lx * b1[c] + ly * b2[c] + lz * w[c];
        }
    }
}

/* Labels from the plain method: hit* = a crossing exists, m* = mu* / l, mu* = t_perp - D*
 * (Eq. 2 inverted, as the paper converts NeRF depth to mu for supervision). */
void orc_train_labels(const orc_scene *sc, int type, int n, const double *o, const double *d,
                      int march_n, int march_b, double *m_star, int *hit_star)
{
    const orc_type *t = &sc->types[type];
    for (int k = 0; k < n; ++k) {
        double ol[3], dl[3], bd[4];
        for (int c = 0; c < 3; ++c) { ol[c] = o[3 * k + c]; dl[c] = d[3 * k + c]; }
        normalize3(dl);
        m_star[k] = 0.0;
        hit_star[k] = 0;
        if (!orc_bound(ol, dl, t->rb, bd)) continue;
        int hit;
        double D = orc_march_depth(sc, type, ol, dl, bd[0], bd[1], march_n, march_b, &hit);
        if (!hit) continue;
        hit_star[k] = 1;
        m_star[k] = (bd[2] - D) / t->rb;
    }
}

/* Loss (regression form of Eq. 6, reading for a "depth + hit logit" network):
 *   L = mean over labelled hits of (m - m*)^2 + 0.1 * mean over all rays of BCE(a, hit*).
 * grad receives dL/dtheta in the packed layout.  Returns L. */
double orc_nedf_loss_grad(const orc_scene *sc, int type, int n, const double *o, const double *d,
                          const double *m_star, const int *hit_star, double *grad, int quant)
{
    const orc_type *t = &sc->types[type];
    int dims[64], nl = nedf_dims(t, dims), maxd = 0;
    for (int l = 0; l <= nl; ++l) maxd = dims[l] > maxd ? dims[l] : maxd;
    size_t np = 0;
    for (int l = 0; l < nl; ++l) np += (size_t)dims[l] * dims[l + 1] + dims[l + 1];
    memset(grad, 0, sizeof(double) * np);
    double *act = (double *)malloc(sizeof(double) * (nl + 1) * maxd);  /* layer inputs */
    double *pre = (double *)malloc(sizeof(double) * (nl + 1) * maxd);  /* pre-activations */
    double *dlt = (double *)malloc(sizeof(double) * maxd), *dnx = (double *)malloc(sizeof(double) * maxd);
    int n_hit = 0;
    for (int k = 0; k < n; ++k) n_hit += hit_star[k] != 0;
    double loss = 0.0;
    for (int k = 0; k < n; ++k) {
        double ol[3], dl[3], bd[4];
        for (int c = 0; c < 3; ++c) { ol[c] = o[3 * k + c]; dl[c] = d[3 * k + c]; }
        normalize3(dl);
        if (!orc_nedf_features(ol, dl, t->rb, act, bd)) continue;
        /* forward with saved activations */
        const double *p = t->nedf_w;
        for (int l = 0; l < nl; ++l) {
            int fi = dims[l], fo = dims[l + 1];
            for (int u = 0; u < fo; ++u) {
                double acc = 0.0;
                for (int i = 0; i < fi; ++i) {
                    double wv = p[(size_t)u * fi + i], av = act[l * maxd + i];
                    if (quant == ORC_QUANT_BF16) { wv = orc_round_bf16(wv); av = orc_round_bf16(av); }
                    acc += wv * av;
                }
                acc += p[(size_t)fi * fo + u];
                pre[(l + 1) * maxd + u] = acc;
                act[(l + 1) * maxd + u] = (l + 1 < nl) ? dmax(acc, 0.0) : acc;
            }
            p += (size_t)fi * fo + fo;
        }
        double m = act[nl * maxd + 0], a = act[nl * maxd + 1];
        double al = hit_star[k] ? 1.0 : 0.0;
        double bce = dmax(a, 0.0) - al * a + log1p(exp(-fabs(a)));
        loss += 0.1 * bce / n;
        dlt[0] = 0.0;
        if (hit_star[k]) {
            loss += (m - m_star[k]) * (m - m_star[k]) / n_hit;
            dlt[0] = 2.0 * (m - m_star[k]) / n_hit;
        }
        dlt[1] = 0.1 * (1.0 / (1.0 + exp(-a)) - al) / n;
        /* backward: dW = delta x input^T, db = delta, d input = W^T delta masked by ReLU */
        size_t off[64];
        off[0] = 0;
        for (int l = 0; l < nl; ++l) off[l + 1] = off[l] + (size_t)dims[l] * dims[l + 1] + dims[l + 1];
        for (int l = nl - 1; l >= 0; --l) {
            int fi = dims[l], fo = dims[l + 1];
            const double *W = t->nedf_w + off[l];
            double *gW = grad + off[l], *gb = grad + off[l] + (size_t)fi * fo;
            for (int u = 0; u < fo; ++u) {
                for (int i = 0; i < fi; ++i) {
                    double av = act[l * maxd + i];
                    if (quant == ORC_QUANT_BF16) av = orc_round_bf16(av);
                    gW[(size_t)u * fi + i] += dlt[u] * av;
                }
                gb[u] += dlt[u];
            }
            if (l == 0) break;
            for (int i = 0; i < fi; ++i) {
                double acc = 0.0;
                for (int u = 0; u < fo; ++u) {
                    double wv = W[(size_t)u * fi + i];
                    if (quant == ORC_QUANT_BF16) wv = orc_round_bf16(wv);
                    acc += wv * dlt[u];
                }
                dnx[i] = pre[l * maxd + i] > 0.0 ? acc : 0.0;
            }
            memcpy(dlt, dnx, sizeof(double) * fi);
            /* BF16 training (reading 29): the error signal of a hidden layer enters its weight
             * product, its bias sum and the next input-gradient product as a BF16 operand; the
             * output layer's (the loss derivative) stays unrounded. */
            if (quant == ORC_QUANT_BF16)
                for (int i = 0; i < fi; ++i) dlt[i] = orc_round_bf16(dlt[i]);
        }
    }
    free(act); free(pre); free(dlt); free(dnx);
    return loss;
}

/* Adam (Kingma & Ba 2015) with bias correction; t counts from 1. */
void orc_adam(int64_t n, double *theta, const double *g, double *m, double *v, int t, double lr,
              double b1, double b2, double eps)
{
    double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        theta[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Supervision by a generic radiance field's density (Section "Intersection network": the NeDF  */
/* is supervised with a pre-trained NeRF through Eq. 5; here any density network)               */
/* ------------------------------------------------------------------------------------------ */
/* sigma(x) = ReLU(o), o the output of the density MLP on the position encoded with 10
 * frequencies (NeRF's density activation). */
double orc_density_net(const double *w, int hidden, int width, const double x[3])
{
    int dims[66];
    dims[0] = 63;
    for (int l = 1; l <= hidden; ++l) dims[l] = width;
    dims[hidden + 1] = 1;
    double f[63], y;
    orc_posenc(x, 3, 10, f);
    orc_mlp(w, hidden + 1, dims, f, &y, ORC_QUANT_NONE);
    return dmax(y, 0.0);
}

/* Labels of n rays (o, d in the object's local frame): n_samples midpoints t_i of the chord
 * [t_e, t_x] through the bound, spacing delta; alpha_i = 1 - exp(-sigma(o + t_i d) delta),
 * T_i = prod_{j<i} (1 - alpha_j), w_i = T_i alpha_i (Eq. 5's weights).  Readings: the label depth
 * is Eq. 5 normalised by the ray's opacity A = sum w_i (the expected termination depth given a
 * termination inside the bound; Eq. 5 itself is the unnormalised sum), and the hit label is
 * A > 0.5.  m* = (t_perp - D) / rb (Eq. 2 inverted); rays missing the bound get A = 0. */
void orc_density_labels(const double *w, int hidden, int width, double rb, int n_samples, int n,
                        const double *o, const double *d, double *m_star, int *hit_star, double *opacity)
{
    for (int k = 0; k < n; ++k) {
        double ol[3], dl[3], bd[4];
        for (int c = 0; c < 3; ++c) { ol[c] = o[3 * k + c]; dl[c] = d[3 * k + c]; }
        normalize3(dl);
        m_star[k] = 0.0;
        hit_star[k] = 0;
        opacity[k] = 0.0;
        if (!orc_bound(ol, dl, rb, bd)) continue;
        const double delta = (bd[1] - bd[0]) / n_samples;
        double T = 1.0, A = 0.0, Dw = 0.0;
        for (int i = 0; i < n_samples; ++i) {
            const double t = bd[0] + (i + 0.5) * delta;
            double x[3];
            for (int c = 0; c < 3; ++c) x[c] = ol[c] + t * dl[c];
            const double alpha = 1.0 - exp(-orc_density_net(w, hidden, width, x) * delta);
            const double wi = T * alpha;
            A += wi;
            Dw += wi * t;
            T *= 1.0 - alpha;
        }
        opacity[k] = A;
        if (A > 0.5) {
            hit_star[k] = 1;
            m_star[k] = (bd[2] - Dw / A) / rb;
        }
    }
}
