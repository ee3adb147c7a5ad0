/* FP64 CPU oracle of the NeDF composition render path (arXiv 2308.04669).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA path; it is never part of it.
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference leg may load it.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * Conventions (inputs are produced by the seeded generator, rounded to float32, then widened):
 *   - An object type is an analytic signed-distance shape inside a bound sphere of radius rb,
 *     with density sigma(x) = sigma_max / (1 + exp(sdf(x) / sdf_width)).
 *   - An instance maps local q to world v = s * R * q + T (R row-major 3x3).  Section
 *     "Manipulating Objects": rays, not sample points, are taken into the local frame.
 *   - A packed MLP holds, layer after layer, W[out][in] row-major then b[out].  Hidden layers
 *     use ReLU, the last layer is linear.
 *   - Pixel p = j * W + i (row j from the top).
 */
#ifndef NEDF_ORACLE_H
#define NEDF_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_SPHERE = 0, ORC_TORUS, ORC_BOX, ORC_CAPSULE, ORC_ROUNDCONE, ORC_TWOSPHERE,
       ORC_TWISTTORUS, ORC_OCTA };
enum { ORC_DEPTH_MLP = 0, ORC_DEPTH_EXACT = 1, ORC_DEPTH_MARCH = 2 };
/* NONE: double throughout.  BF16: every layer's weights and inputs rounded to BF16.  FP8: the
 * first layer as BF16; every later hidden layer's weights as s_l * E4M3(W / s_l) with s_l the
 * power of two that puts max|W| in (224, 448]; every hidden activation rounded to E4M3; the output
 * layer's weights rounded to BF16.  Sums and biases stay in double in every mode. */
enum { ORC_QUANT_NONE = 0, ORC_QUANT_BF16 = 1, ORC_QUANT_FP8 = 2 };

/* The paper's intersection network (Section "Intersection network", Appendix A): 16 points per
 * ray, 10 encoding frequencies (16 x 63 = 1008 inputs), a 256-wide head, 16 residual blocks, a
 * two-level classifier of 64 coarse and 128 fine bins.  Packed weights, W[out][in] then b[out]:
 * head 1008 -> 256; per block W1, b1, W2, b2 (256 -> 256 each); tail A 256 -> 65 (row 0 the hit
 * logit, rows 1..64 the coarse bins); tail B 256 -> 128 (the fine bins). */
enum { ORC_CLS_PTS = 16, ORC_CLS_FREQ = 10, ORC_CLS_IN = 1008, ORC_CLS_W = 256, ORC_CLS_BLOCKS = 16,
       ORC_CLS_NC = 64, ORC_CLS_NF = 128, ORC_CLS_OUT = 1 + 64 + 128 };
enum { ORC_ARCH_REGRESSION = 0, ORC_ARCH_CLASSIFIER = 1 };

typedef struct {
    int kind;
    double params[8];
    double rb;
    double albedo[3];
    int nedf_hidden, nedf_width;
    const double *nedf_w;
    int nerf_hidden, nerf_width; /* nerf_hidden == 0: constant albedo colour */
    const double *nerf_w;
    int nedf_arch;               /* ORC_ARCH_*: the regression MLP above or the classifier */
    const double *nedf_wq;       /* classifier: nedf_w with every weight (not bias) rounded to BF16
                                    (orc_cls_round_bf16), used by the BF16 mode */
} orc_type;

typedef struct {
    int W, H;
    double eye[3], target[3], fov_deg;
    int n_lights;
    const double *lights; /* [n_lights][3] */
    int n_types;
    const orc_type *types;
    int n_inst;
    const int *inst_type;
    const double *inst_R; /* [n][9] */
    const double *inst_T; /* [n][3] */
    const double *inst_s; /* [n] */
    int n_shade;
    double shade_half, beta, eps, sigma_max, sdf_width;
    const int *light_parallel; /* [n_lights] or NULL: nonzero = a parallel light, lights[l] its
                                  travel direction (the "parallel light sources" of Section 1) */
} orc_scene;

typedef struct {
    int depth_mode;        /* ORC_DEPTH_* */
    int march_n, march_b;  /* MARCH mode, and the fallback march */
    int quant;             /* ORC_QUANT_*: rounding applied to every layer's operands */
    double fallback_conf;  /* MLP mode: march the pair when max(p,1-p) < this (0 = never) */
    int refine_steps;      /* MLP mode: density bisection steps around the NeDF depth (0 = off) */
    int n_threads;
    int outlier_resample;  /* MLP mode, with refine_steps > 0: a NeDF hit whose window [D-h, D+h]
                              holds no density crossing is re-answered by the plain method */
    int shade_resample;    /* Step-2 outlier resampling (Section "Deferred Shading", "rs"): a shaded
                              pixel whose largest density over its n_shade samples is below
                              shade_sigma_min is re-rendered by the plain method's volume rendering
                              (this many samples per pair); 0 = off */
    double shade_sigma_min;
    int miss_check;        /* MLP mode: a miss kept by the confidence test is checked at this many
                              midpoints of its bound chord and re-answered by the plain method when
                              the density reaches the half level at one (0 = off) */
} orc_opts;

/* Geometry and encoding */
double orc_sdf(int kind, const double *params, const double x[3]);
double orc_density(const orc_scene *sc, int type, const double x[3]);
void orc_camera_ray(const orc_scene *sc, int i, int j, double o[3], double d[3]);
void orc_to_local(const orc_scene *sc, int inst, const double o[3], const double d[3],
                  double ol[3], double dl[3]);
int orc_bound(const double ol[3], const double dl[3], double rb, double out4[4]);
int orc_posenc(const double *x, int n, int n_freq, double *out);
int orc_nedf_features(const double ol[3], const double dl[3], double rb, double *feat78,
                      double out4[4]);

/* Networks */
void orc_mlp(const double *w, int n_layers, const int *dims, const double *x, double *y, int quant);
/* Distance from v to the nearest rounding boundary of BF16 (fmt 0) or E4M3 (fmt 1). */
double orc_round_margin(double v, int fmt);
/* orc_mlp plus the row's rounding knife edge: the smallest distance of a BF16 / E4M3-rounded value
 * to its rounding boundary relative to the magnitude of the sum that produced it, max(|v|, 1/4) for
 * an input feature (INFINITY in the unrounded mode). */
double orc_mlp_qmargin(const double *w, int n_layers, const int *dims, const double *x, double *y, int quant);
/* orc_mlp with value flip_idx (inputs first, then each hidden layer's outputs; -1 none) rounded to
 * its other neighbour; the n_cand values nearest to a rounding boundary (relative margin,
 * ascending) are listed in cand_idx / cand_margin. */
void orc_mlp_flip(const double *w, int n_layers, const int *dims, const double *x, double *y, int quant,
                  int flip_idx, int n_cand, int *cand_idx, double *cand_margin);
/* orc_mlp with two values (flip_a, flip_b) rounded to their other neighbours. */
void orc_mlp_flip2(const double *w, int n_layers, const int *dims, const double *x, double *y, int quant, int flip_a,
                   int flip_b);
/* orc_mlp with the n_flips values whose indices are listed in flips rounded to their other
 * neighbours (several near-ties of one row may each fall on either side). */
void orc_mlp_flipset(const double *w, int n_layers, const int *dims, const double *x, double *y, int quant,
                     int n_flips, const int *flips);
double orc_round_bf16(double x);
double orc_round_e4m3(double x);
double orc_fp8_scale(double max_abs);

/* The classifier intersection network */
int64_t orc_cls_param_count(void);
int orc_cls_features(const double ol[3], const double dl[3], double rb, double *feat1008, double out4[4]);
void orc_cls_round_bf16(const double *w, double *wq);
void orc_cls_forward(const double *w, const double *x, double *logits, int quant);
void orc_cls_segment(double m, int *c, int *f);
double orc_cls_decode(const double *logits, double *m, double *a, int *c, int *f);
double orc_cls_loss_grad(const double *w, int n, const double *x, const double *m_star,
                         const int *hit_star, double *grad);

/* One (ray, instance) query: returns 1 on hit; out6 = {Dl, m, a, te, tx, tperp} */
int orc_query(const orc_scene *sc, const orc_opts *op, int inst, const double o[3],
              const double d[3], double out6[6], double *margin);
/* orc_query with its knife-edge diagnostics: diag = {margin, dmargin, dspread}.  dmargin is the
 * smallest margin of the plain method's and the refinement's inside tests whose consequence (how
 * far the depth moves if the test goes the other way: half the bracket for a bisection step,
 * unbounded otherwise) is at least `need` (local length); a test's margin is |sdf| at its point,
 * less the network-rounding depth shift, over |o_local| + |t| + rb (INFINITY when no such test
 * ran).  dspread is the local depth shift a single BF16 / E4M3 rounding flip of the network can
 * cause. */
int orc_query_diag(const orc_scene *sc, const orc_opts *op, int inst, const double o[3], const double d[3],
                   double out6[6], double diag[3], double need);
double orc_exact_depth(int kind, const double *params, const double ol[3], const double dl[3],
                       double te, double tx, int *hit);
double orc_march_depth(const orc_scene *sc, int type, const double ol[3], const double dl[3],
                       double te, double tx, int n, int b, int *hit);

/* Shading quadrature over n samples (Eq. 8 with the sample window): rgba = (sum T a c, sum T a) */
void orc_composite_samples(int n, const double *sigma, const double *rgb, double world_delta,
                           double rgba[4]);

/* Steps 1-3 of Algorithm 1 / Algorithm 2 for a list of pixels.  Besides the buffers, per pixel:
 * gap      distance from the nearest hit to the next one, less the depth shift that single
 *          network-rounding flips can cause on either (BF16 / E4M3 modes);
 * pmargin  smallest distance of a Step-1 decision (cull, hit logit, D > 0, confidence, depth-check
 *          window) from its threshold;
 * smargin  the same for the shadow tests of Step 3;
 * dmargin  relative margin (see orc_query_diag) of the most critical depth test (the plain
 *          method's and the refinement's inside tests) among those that can change the pixel:
 *          all of the winner's, those of another hit or a shadow query whose consequence reaches
 *          the winner or the shadow test, and the unbounded ones of misses.  When `alt` is given
 *          and that margin is below 1e-6, the pixel is rendered again with that test taken the
 *          other way into alt[12 k ..] = {depth, id (-1: none), rgba[4], shadow, out[4], 1}
 *          (NaN and 0 otherwise), and dmargin is the second most critical test's margin. */
int orc_render(const orc_scene *sc, const orc_opts *op, int64_t n_px, const int64_t *px,
               double *depth, uint32_t *id, double *gap, double *pmargin, double *rgba,
               double *shadow, double *smargin, double *out, double *shade_smax, double *dmargin,
               double *alt);

/* Steps 2-3 (Eq. 8 shading, Algorithm 2 shadows, the composite) of pixels px given each pixel's
 * winning instance id and world depth (id 0xFFFFFFFF: no hit): the oracle's answer to another
 * implementation's Step-1 result, so that its Steps 2-3 can be checked exactly given that result.
 * smargin as in orc_render. */
int orc_steps23(const orc_scene *sc, const orc_opts *op, int64_t n_px, const int64_t *px, const uint32_t *id,
                const double *depth, double *rgba, double *shadow, double *smargin, double *out);

/* Plain method: dense front-to-back volume rendering with n samples per (ray, instance).
 * vmargin (may be NULL): per pixel, the smallest cull-discriminant / rb^2 and entry-distance
 * difference between consecutive pairs (the decisions a rounding change could flip). */
int orc_volume_render(const orc_scene *sc, const orc_opts *op, int n_samples, int64_t n_px,
                      const int64_t *px, double *rgba, double *vmargin);

/* Learned part */
uint64_t orc_splitmix64(uint64_t seed, uint64_t index);
void orc_train_rays(double rb, uint64_t seed, int64_t first, int n, double *o, double *d);
void orc_train_labels(const orc_scene *sc, int type, int n, const double *o, const double *d,
                      int march_n, int march_b, double *m_star, int *hit_star);
/* Loss (the regression form of Eq. 6, reading 18) and its gradient by hand.  quant = BF16 is the
 * BF16 training of reading 29: forward operands (weights, layer inputs) rounded to BF16; in the
 * backward pass the weights and the saved activations are the BF16 values and each hidden layer's
 * error signal is rounded to BF16 before its weight product, bias sum and input-gradient product;
 * the loss derivative at the output stays unrounded. */
double orc_nedf_loss_grad(const orc_scene *sc, int type, int n, const double *o, const double *d,
                          const double *m_star, const int *hit_star, double *grad, int quant);
void orc_adam(int64_t n, double *theta, const double *g, double *m, double *v, int t, double lr,
              double b1, double b2, double eps);

/* Supervision by a generic radiance field's density network (plugin mode): sigma(x) =
 * ReLU(MLP(gamma_10(x))), the MLP [63, width x hidden, 1] in the packed layout; labels from Eq. 5
 * over n_samples midpoints of the chord through the bound (see orc_density_labels). */
double orc_density_net(const double *w, int hidden, int width, const double x[3]);
void orc_density_labels(const double *w, int hidden, int width, double rb, int n_samples, int n,
                        const double *o, const double *d, double *m_star, int *hit_star, double *opacity);

#ifdef __cplusplus
}
#endif
#endif
