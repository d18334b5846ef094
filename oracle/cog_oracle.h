/*
 * cog_oracle.h -- plain, slow FP64 CPU oracle for the per-pixel
 * Rejection-Cascade of Gaussians (CoG) background-subtraction step of
 * Kiran, Das and Yogamani, "Rejection-Cascade of Gaussians: real-time
 * adaptive background subtraction framework" (arXiv 1705.09339).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library in the package; the two
 * meet only through the seeded synthetic-video generator (cogsynth), which
 * holds none of the method's arithmetic.
 *
 * Every routine follows the paper's passage it names:
 *   - scene prior (kernel density over the N training frames, quantised to
 *     255 or, with kde_bits = 4, to 15 levels of its peak, and entering the
 *     confidence as the fraction q / Q of the peak): Sec. 2, "Scene Prior in
 *     Background Model" and Eq. 2;
 *   - residue classes -> confidence weights: Sec. 2, "Determining Learning
 *     Rate Hyper-parameters";
 *   - Stauffer-Grimson mixture update: Eq. 2 (with the garbled variance line
 *     read as the usual squared-residual update, rho = the effective rate);
 *   - confidence C = a P + b dI + g M: Sec. 2, "Confidence Measure";
 *   - cascade CHP -> running Gaussian average -> ordered Gaussians, prior
 *     nullified, active-level-only adaptation, illumination counter:
 *     Sec. 2, "Cascade of Gaussians CoG";
 *   - ORC_PERCHAN, per-channel independent mixtures (the independence of
 *     the R, G, B channels Sec. 2 assumes for the prior, applied to the
 *     mixture): each channel ranks, matches and updates its own K 1-D
 *     components with its own weights; a pixel is background iff every
 *     channel is;
 *   - ORC_MODE1, the Fig. 1 reading of the cascade (CHP -> mode 1 -> the
 *     other modes): stage 1 tests and adapts a copy of the mixture's
 *     rank-1 mode; on the transition to stage 2 the copy is written back
 *     into that mode ("during a transition the parameters are updated",
 *     Sec. 2), Eq. 2 runs, and the copy then follows the new rank-1 mode;
 *   - spatio-temporal grouping (training side): Sec. 2, "Clustering Similar
 *     Background - Spatio-Temporal Grouping", its steps 1-6 and Eq. 3.
 * The readings taken where the text is silent or garbled are listed in the
 * repository's design notes and restated beside the code below.
 *
 * Parity status: the KDE, residue weights, the mixture update, weight
 * normalisation, the static-pixel variance decay, the step absorption time,
 * the constant-input confidence recursion, the flags-off == plain-GMM
 * identity and the illumination response are pinned by closed forms and
 * invariants in the CPU tests, and so are the grouping features (constant
 * and two-level pixels worked by hand), the K-means fixed point and the
 * Eq. 3 cores (brute force).  The overall behaviour of the full cascade on
 * natural video has no printed worked example in the paper: beyond those
 * pins it is "parity unpinned".
 */
#ifndef COG_ORACLE_H
#define COG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* stage switches */
#define ORC_FD    1u   /* stage 0: frame difference / consistent-hypothesis propagation */
#define ORC_RGA   2u   /* stage 1: running Gaussian average                             */
#define ORC_CONF  4u   /* confidence-driven rates, thresholds and halting                */
#define ORC_ILLUM 8u   /* abrupt-illumination counter and response                       */
#define ORC_SAMPLE 16u /* confidence-based temporal sampling                             */
#define ORC_MODE1 32u  /* stage 1 is the mixture's rank-1 mode (Fig. 1 reading)        */
#define ORC_PERCHAN 64u /* per-channel independent mixtures (own weights per channel)    */

/* near-threshold record bits (one byte per pixel and frame) */
#define ORC_NEAR_FD    1u  /* D vs tau_fd (0.5 + C)            */
#define ORC_NEAR_RGA   2u  /* t_r vs 1                         */
#define ORC_NEAR_MATCH 4u  /* some evaluated t_k vs 1          */
#define ORC_NEAR_BGSET 8u  /* weight ranked before match vs T  */
#define ORC_NEAR_RANK 16u  /* two adjacent rank keys nearly tie */
#define ORC_NEAR_HALT 32u  /* C vs c_halt                      */
#define ORC_NEAR_SKIP 64u  /* C vs c_skip                      */

/* stage codes written to the stage map */
#define ORC_ST_FD     0
#define ORC_ST_RGA    1
#define ORC_ST_GMM_BG 2
#define ORC_ST_FG     3
#define ORC_ST_ILLUM  4
#define ORC_ST_SKIP   5   /* not sampled this frame: label carried       */

typedef struct {
    int width, height;  /* pixels are numbered p = y*width + x          */
    int K;              /* Gaussians per pixel, 1..8                    */
    double alpha;       /* base learning rate                           */
    double lambda;      /* match threshold in standard deviations       */
    double T_bg;        /* background weight fraction T                 */
    double w_init;      /* weight of a newly created component          */
    double var_init, var_min, var_max;
    double tau_fd;      /* frame-difference threshold at C = 0.5        */
    double eta;         /* confidence smoothing rate                    */
    double c_halt;      /* confidence at which RGA updates stop         */
    double w_illum;     /* weight given on an illumination change       */
    double c_skip;      /* sampling: confidence at which a pixel is only
                           processed every skip_period frames           */
    int q_null;         /* prior nullified below q_null / 255 of peak   */
    int kde_bw;         /* kernel bandwidth in grey levels              */
    int r1, r2;         /* residue class bounds                         */
    int illum_permille; /* illumination threshold, per mille of pixels  */
    int skip_period;    /* sampling period S (>= 1)                     */
    unsigned flags;     /* ORC_* switches                               */
    int kde_bits;       /* prior levels: 8 (0..255) or 4 (0..15)        */
} orc_params;

/* Model state, all arrays owned by the caller. P = width*height. */
typedef struct {
    double  *w;      /* [P][K]       mixture weights                    */
    double  *mu;     /* [P][K][3]    means                              */
    double  *var;    /* [P][K][3]    per-channel variances              */
    double  *rga_m;  /* [P][3]       running-average mean               */
    double  *rga_v;  /* [P][3]       running-average variance           */
    double  *conf;   /* [P]          confidence C                       */
    uint8_t *label;  /* [P]          previous label, 0 = BG, 1 = FG     */
    uint8_t *prev;   /* [P][3]       previous frame J                   */
    uint8_t *kde;    /* [P][3][256]  peak-normalised prior q_c[v], one
                                     level per byte (0..2^kde_bits - 1)  */
    uint8_t *qa;     /* [P]          static-class weight, of 255        */
    uint8_t *qb;     /* [P]          dynamic-class weight, of 255       */
    int64_t *illum;  /* [2]          [0]: pixels that reached the GMM stage in
                                     the previous frame; [1]: frames applied
                                     since training                     */
    uint8_t *top;    /* [P]          with ORC_MODE1: the mixture component the
                                     running average mirrors            */
    double  *wc;     /* [P][3][K]    with ORC_PERCHAN: each channel's own
                                     mixture weights (w is then unused) */
} orc_state;

typedef struct {
    int64_t n_stage[6];   /* pixels per ORC_ST_* code                */
    int64_t n_gmm;        /* pixels that reached the GMM stage       */
    int32_t illum_flag;   /* flag used for this frame                */
    int32_t pad;
} orc_stats;

/* Integer Gaussian weights g[d] = round(65536 exp(-d^2 / (2 bw^2))),
 * d = 0..3bw.  Writes 3bw+1 entries when cap allows; returns 3bw, or -1. */
int orc_kde_weights(int bw, int64_t *g, int cap);

/* Training over frames[N][P][3] (N >= 2): KDE prior, residue weights,
 * mixture warm-up, running-average and confidence initialisation. */
int orc_train(const orc_params *pr, const uint8_t *frames, int N, orc_state *s);

/* orc_train that also records, per pixel, the OR of the near-threshold bits
 * (ORC_NEAR_*) of every warm-up decision over frames 1..N-1, plus
 * ORC_NEAR_RANK when the top-ranked mode that seeds the running average
 * nearly ties another; near[P] may be NULL. */
int orc_train_near(const orc_params *pr, const uint8_t *frames, int N, orc_state *s, uint8_t *near);

/* One test frame through the cascade.  frame[P][3]; mask[P] (0/255);
 * stage[P] and near[P] are optional (NULL skips them). */
int orc_apply(const orc_params *pr, orc_state *s, const uint8_t *frame,
              uint8_t *mask, uint8_t *stage, uint8_t *near, orc_stats *st);

/* One frame of the textbook Stauffer-Grimson mixture (the paper's
 * comparison baseline), written in the background-set form: rank, find the
 * first b components whose weights exceed T, match, update.  Rate = alpha. */
int orc_plain_gmm(const orc_params *pr, double *w, double *mu, double *var,
                  const uint8_t *frame, uint8_t *mask);

/* Number of OpenMP threads the oracle uses (1 without OpenMP), and a way
 * to change it (n >= 1) for timing. */
int orc_threads(void);
void orc_set_threads(int n);

/* Spatio-temporal grouping features (Sec. 2, "Clustering Similar
 * Background"): the mixture warm-up of orc_train replayed over
 * frames[N][P][3]; after each update at frames 1..N-1 the dominant mode
 * (largest omega^2 / vbar, lowest index on ties) gives its mean variance
 * vbar and weight omega.  code_v[p] = round(64 sd(vbar)), code_w[p] =
 * round(65536 sd(omega)), population standard deviations over the N-1
 * updates, saturated at 65535.  Not defined with ORC_PERCHAN. */
int orc_group_features(const orc_params *pr, const uint8_t *frames, int N,
                       uint16_t *code_v, uint16_t *code_w);

/* Grouping result: K-means labels and the Eq. 3 cores. */
typedef struct {
    int32_t iterations;     /* Lloyd steps until no label changed (max_iter if none) */
    int32_t converged;      /* 1: the labels settled within max_iter                 */
    int64_t n[3];           /* pixels per cluster                                    */
    int64_t n_core[3];      /* of them inside the Eq. 3 band on both features       */
    int64_t s1[3][2];       /* per cluster: sums of code_v, code_w                   */
    int64_t s2[3][2];       /*              sums of their squares                    */
    double centroid[3][2];  /* member means of the codes                             */
    double sd[3][2];        /* member standard deviations of the codes               */
    double w1[3];           /* orc_group_params: mean over the core of the dominant  */
    double mu1[3][3];       /* mode's weight, means and mean variance                */
    double v1[3];
    int64_t n_near;         /* assignments, over all steps, that were near a tie     */
} orc_group_out;

/* Steps 4-5: K-means, K = 3, over (code_v, code_w) scaled by their
 * standard deviations over all P pixels (1 for a constant feature), first
 * centroids at mean - sd, mean, mean + sd (sd = 0 for a constant feature:
 * the centroids start on its one value), an empty cluster keeping its
 * centroid, ties to the lower cluster, the distance in FP64; at most
 * max_iter Lloyd steps after the first assignment (max_iter >= 0).  Then
 * each pixel whose two codes lie strictly within its cluster's mean +-
 * standard deviation (Eq. 3) is a core pixel.  labels[p] = cluster | 0x80
 * for a core pixel.  The run is composed of the three steps below. */
int orc_group_cluster(int64_t P, const uint16_t *code_v, const uint16_t *code_w, int max_iter,
                      uint8_t *labels, orc_group_out *out);

/* The feature scales sd[2] (spread over all pixels, 1 for a constant
 * feature) and the first centroids c[3][2]. */
int orc_group_init(int64_t P, const uint16_t *code_v, const uint16_t *code_w, double c[3][2], double sd[2]);

/* One Lloyd update: c[j] <- the mean codes of the pixels labelled j
 * (labels & 0x7f); a cluster with no pixel keeps c[j]. */
int orc_group_centroids(int64_t P, const uint16_t *code_v, const uint16_t *code_w, const uint8_t *labels,
                        double c[3][2]);

/* One assignment: labels[p] = the nearest centroid in the scaled FP64
 * distance, ties to the lower cluster.  near (nullable) gets 1 where the
 * two nearest distances are within 1e-5 relative of each other or within
 * twice the bound on a single-precision evaluation's error of them (the
 * centroid and scales rounded to single precision, every operation
 * rounded): there the decision may go either way in an implementation that
 * computes the distance in single precision.  Returns the number of near
 * pixels, or -1 for bad arguments. */
int64_t orc_group_assign(int64_t P, const uint16_t *code_v, const uint16_t *code_w, const double c[3][2],
                         const double sd[2], uint8_t *labels, uint8_t *near);

/* Step 5 on given labels (the core bit of labels is ignored and
 * rewritten): per cluster the count, the sums of the codes and of their
 * squares, the member means and standard deviations, and the Eq. 3 core
 * (labels[p] |= 0x80, n_core). */
int orc_group_cores(int64_t P, const uint16_t *code_v, const uint16_t *code_w, uint8_t *labels, orc_group_out *out);

/* Step 6: per cluster, the mean over its core pixels of the trained
 * state's dominant mode (the one orc_train gave the running average):
 * weight, per-channel means and mean variance, into out->w1, mu1, v1. */
int orc_group_params(const orc_params *pr, const orc_state *s, const uint8_t *labels, orc_group_out *out);

#ifdef __cplusplus
}
#endif
#endif
