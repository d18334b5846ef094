/*
 * cog_oracle.c -- FP64 CPU oracle of the Cascade-of-Gaussians step.
 *
 * TEST INFRASTRUCTURE ONLY (see cog_oracle.h): nothing in the product path
 * may link, load or call it.  It is deliberately plain: one pixel at a
 * time, the steps in the order the paper states them, no blocking, no
 * fusion.  OpenMP only distributes independent pixels over threads; it does
 * not change any arithmetic or its order.
 */
#include "cog_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NEAR_REL 1e-4
#define KMAX 8

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

static int near_rel(double x, double thr)
{
    return fabs(x - thr) <= NEAR_REL * fabs(thr);
}

static double clampd(double x, double lo, double hi)
{
    return x < lo ? lo : (x > hi ? hi : x);
}

static int check_params(const orc_params *pr)
{
    if (!pr || pr->width <= 0 || pr->height <= 0) return -1;
    if (pr->K < 1 || pr->K > KMAX) return -1;
    if (!(pr->var_min > 0.0) || pr->var_max < pr->var_min) return -1;
    if (pr->kde_bw < 1 || pr->kde_bw > 32) return -1;
    if (pr->kde_bits != 8 && pr->kde_bits != 4) return -1;
    if ((pr->flags & ORC_SAMPLE) && pr->skip_period < 1) return -1;
    if ((pr->flags & ORC_PERCHAN) && (pr->flags & ORC_MODE1)) return -1;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Scene prior: Sec. 2 "Scene Prior in Background Model".  A kernel      */
/* density over the N training values of each pixel and channel, with a  */
/* Gaussian kernel K_sigma of bandwidth bw, independent R, G, B.  The     */
/* density is evaluated on the 256 grey levels in integer arithmetic:     */
/*   k[v] = sum_u h[u] g[v-u],  g[d] = round(2^16 exp(-d^2/(2 bw^2)))     */
/* truncated at |d| <= 3 bw, then normalised to its peak and quantised */
/* to Q = 2^kde_bits - 1 levels (255 for the 8-bit prior, 15 for 4-bit):  */
/*   q[v] = (Q k[v] + M/2) div M,  M = max_v k[v].                        */
/* ------------------------------------------------------------------ */
int orc_kde_weights(int bw, int64_t *g, int cap)
{
    if (bw < 1 || !g || cap < 3 * bw + 1) return -1;
    for (int d = 0; d <= 3 * bw; d++) {
        double x = 65536.0 * exp(-(double)(d * d) / (2.0 * bw * bw));
        g[d] = (int64_t)floor(x + 0.5);
    }
    return 3 * bw;
}

static void kde_one(const uint8_t *frames, int N, int64_t P, int64_t p, int c,
                    const int64_t *g, int R, int64_t Q, uint8_t *q)
{
    int64_t h[256];
    int64_t k[256];
    memset(h, 0, sizeof h);
    for (int t = 0; t < N; t++)
        h[frames[((int64_t)t * P + p) * 3 + c]]++;
    int64_t M = 0;
    for (int v = 0; v < 256; v++) {
        int64_t acc = 0;
        for (int u = (v - R > 0 ? v - R : 0); u <= (v + R < 255 ? v + R : 255); u++) {
            int d = v > u ? v - u : u - v;
            acc += h[u] * g[d];
        }
        k[v] = acc;
        if (acc > M) M = acc;
    }
    for (int v = 0; v < 256; v++)
        q[v] = (uint8_t)((Q * k[v] + M / 2) / M);
}

/* The prior's value at the pixel's colour (Sec. 2, "Confidence Measure" and
 * "Cascade of Gaussians CoG"): the smallest of the three channel levels as a
 * fraction of the peak, q / Q.  The prior is nullified when that fraction
 * is below q_null / 255 (q_null is on the 8-bit scale for either width),
 * decided exactly in integers: 255 q < q_null Q. */
static int prior_nullified(const orc_params *pr, const orc_state *s, int64_t p, const uint8_t *I,
                           double *frac)
{
    const int Q = (1 << pr->kde_bits) - 1;
    int qmin = Q;
    for (int c = 0; c < 3; c++) {
        int q = s->kde[(p * 3 + c) * 256 + I[c]];
        if (q < qmin) qmin = q;
    }
    *frac = (double)qmin / Q;
    return 255 * qmin < pr->q_null * Q;
}

/* ------------------------------------------------------------------ */
/* Residue classes: Sec. 2 "Determining Learning Rate Hyper-parameters". */
/* R_t = I_t - I_{t-1} over the training frames, summarised per pixel by  */
/* the largest absolute channel difference, binned into three classes    */
/* (static/drift <= r1 < oscillating <= r2 < dynamic).  The normalised    */
/* bin frequencies become the confidence weights: a <- static fraction,   */
/* b <- dynamic fraction, g <- the oscillating remainder.                 */
/* ------------------------------------------------------------------ */
static void residue_one(const orc_params *pr, const uint8_t *frames, int N,
                        int64_t P, int64_t p, uint8_t *qa, uint8_t *qb)
{
    int64_t n0 = 0, n1 = 0, n2 = 0;
    for (int t = 1; t < N; t++) {
        int R = 0;
        for (int c = 0; c < 3; c++) {
            int a = frames[((int64_t)t * P + p) * 3 + c];
            int b = frames[((int64_t)(t - 1) * P + p) * 3 + c];
            int d = a > b ? a - b : b - a;
            if (d > R) R = d;
        }
        if (R <= pr->r1) n0++;
        else if (R <= pr->r2) n1++;
        else n2++;
    }
    (void)n1;
    int64_t n = N - 1;
    int64_t a = (255 * n0 + n / 2) / n;
    int64_t b = (255 * n2 + n / 2) / n;
    if (b > 255 - a) b = 255 - a;
    *qa = (uint8_t)a;
    *qb = (uint8_t)b;
}

/* ------------------------------------------------------------------ */
/* Per-pixel cascade: Sec. 2 "Confidence Measure" and "Cascade of       */
/* Gaussians CoG", with the mixture of Eq. 2.                           */
/* ------------------------------------------------------------------ */
typedef struct {
    int stage;       /* ORC_ST_* */
    int reached_gmm; /* counted for the illumination counter */
    uint8_t near;
} px_out;

/* Stage 2 with per-channel independent mixtures (ORC_PERCHAN): channel c
 * ranks its components by w_c^2 / v_c, takes the first in rank order with
 * (I_c - mu_c)^2 / (lambda^2 v_c) < 1, is background iff the weight ranked
 * before it is <= T, and updates its own weights (Eq. 2 per channel); a
 * channel with no match restarts its lowest-ranked component.  The pixel is
 * background iff every channel is.  Returns the label; *Mhat receives the
 * largest per-channel match statistic (1 for an unmatched channel). */
static int stage2_perchan(const orc_params *pr, orc_state *s, int64_t p, const uint8_t *I,
                          double a_eff, int illum_flag, double *Mhat, uint8_t *near, int *illum)
{
    const int K = pr->K;
    const double lam2 = pr->lambda * pr->lambda;
    double *mu = s->mu + p * K * 3;
    double *var = s->var + p * K * 3;
    int chan_fg[3], tgt_c[3], label = 0;
    *Mhat = 0.0;
    for (int c = 0; c < 3; c++) {
        double *w = s->wc + (p * 3 + c) * K;
        double r[KMAX];
        int ord[KMAX];
        for (int k = 0; k < K; k++) r[k] = w[k] * w[k] / var[k * 3 + c];
        for (int k = 0; k < K; k++) ord[k] = k;
        for (int i = 1; i < K; i++) {            /* stable insertion sort */
            int x = ord[i], j = i - 1;
            while (j >= 0 && r[ord[j]] < r[x]) { ord[j + 1] = ord[j]; j--; }
            ord[j + 1] = x;
        }
        for (int i = 0; i + 1 < K; i++) {
            double ra = r[ord[i]], rb = r[ord[i + 1]];
            double mx = ra > rb ? ra : rb;
            if (ra != rb && fabs(ra - rb) <= NEAR_REL * mx) *near |= ORC_NEAR_RANK;
        }
        int m = -1, mpos = -1;
        double tm = 0.0;
        for (int j = 0; j < K; j++) {
            int k = ord[j];
            double d = I[c] - mu[k * 3 + c];
            double tk = d * d / (lam2 * var[k * 3 + c]);
            if (near_rel(tk, 1.0)) *near |= ORC_NEAR_MATCH;
            if (tk < 1.0) { m = k; mpos = j; tm = tk; break; }
        }
        int fgc = 1;
        if (m >= 0) {
            double S = 0.0;
            for (int j = 0; j < mpos; j++) S += w[ord[j]];
            if (near_rel(S, pr->T_bg)) *near |= ORC_NEAR_BGSET;
            fgc = (S <= pr->T_bg) ? 0 : 1;
        }
        const double Mc = (m >= 0) ? (tm < 1.0 ? tm : 1.0) : 1.0;
        if (Mc > *Mhat) *Mhat = Mc;
        int tgt;
        if (m >= 0) {
            for (int k = 0; k < K; k++) w[k] = (1.0 - a_eff) * w[k] + (k == m ? a_eff : 0.0);
            double *pm = &mu[m * 3 + c], *pv = &var[m * 3 + c];
            *pm = *pm + a_eff * (I[c] - *pm);
            double d = I[c] - *pm;
            *pv = clampd((1.0 - a_eff) * (*pv) + a_eff * d * d, pr->var_min, pr->var_max);
            tgt = m;
        } else {
            for (int k = 0; k < K; k++) w[k] = (1.0 - a_eff) * w[k];
            int low = ord[K - 1];
            mu[low * 3 + c] = I[c];
            var[low * 3 + c] = pr->var_init;
            w[low] = pr->w_init;
            tgt = low;
        }
        double sum = 0.0;
        for (int k = 0; k < K; k++) sum += w[k];
        for (int k = 0; k < K; k++) w[k] = w[k] / sum;
        chan_fg[c] = fgc;
        tgt_c[c] = tgt;
        label |= fgc;
    }
    *illum = 0;
    if (illum_flag && label) {
        /* abrupt illumination change: every channel that decided foreground
         * gives its matched or new component the weight w_illum */
        for (int c = 0; c < 3; c++) {
            if (!chan_fg[c]) continue;
            double *w = s->wc + (p * 3 + c) * K;
            double so = 0.0;
            for (int k = 0; k < K; k++) if (k != tgt_c[c]) so += w[k];
            if (so > 0.0) {
                for (int k = 0; k < K; k++)
                    if (k != tgt_c[c]) w[k] = w[k] * (1.0 - pr->w_illum) / so;
                w[tgt_c[c]] = pr->w_illum;
            } else {
                w[tgt_c[c]] = 1.0;
            }
        }
        label = 0;
        *illum = 1;
    }
    if (label == 0) {   /* transition update, channel by channel */
        for (int c = 0; c < 3; c++) {
            s->rga_m[p * 3 + c] = mu[tgt_c[c] * 3 + c];
            s->rga_v[p * 3 + c] = var[tgt_c[c] * 3 + c];
        }
    }
    return label;
}

static px_out cascade_pixel(const orc_params *pr, orc_state *s, int64_t p,
                            const uint8_t *I, int illum_flag, int64_t n)
{
    const int K = pr->K;
    const double lam2 = pr->lambda * pr->lambda;
    const unsigned fl = pr->flags;
    px_out o = {0, 0, 0};

    double *w = s->w + p * K;
    double *mu = s->mu + p * K * 3;
    double *var = s->var + p * K * 3;
    double *rm = s->rga_m + p * 3;
    double *rv = s->rga_v + p * 3;
    uint8_t *J = s->prev + p * 3;

    /* Pre-frame values.  Without the confidence switch every modulation
     * is neutral (C- = 0.5 gives rate alpha and threshold tau_fd). */
    const double Cm = (fl & ORC_CONF) ? s->conf[p] : 0.5;
    const double a_eff = pr->alpha * (1.5 - Cm);
    const int halt = (fl & ORC_CONF) && Cm >= pr->c_halt;
    if ((fl & ORC_CONF) && near_rel(Cm, pr->c_halt)) o.near |= ORC_NEAR_HALT;

    /* Confidence-based temporal sampling (Sec. 2, "Confidence based temporal
     * sampling"): a pixel whose confidence has saturated is looked at only
     * every skip_period frames, in 64-pixel blocks with staggered phases;
     * in between it keeps its label and nothing about it changes. */
    if ((fl & ORC_SAMPLE) && (fl & ORC_CONF)) {
        if (near_rel(Cm, pr->c_skip)) o.near |= ORC_NEAR_SKIP;
        if (Cm >= pr->c_skip && (n + (p >> 6)) % pr->skip_period != 0) {
            o.stage = ORC_ST_SKIP;
            return o;
        }
    }

    int D = 0;
    for (int c = 0; c < 3; c++) {
        int d = I[c] > J[c] ? I[c] - J[c] : J[c] - I[c];
        if (d > D) D = d;
    }
    const double wa = s->qa[p] / 255.0;
    const double wb = s->qb[p] / 255.0;
    const double wg = (255 - s->qa[p] - s->qb[p]) / 255.0;
    const double dhat = D / 255.0;

    int label = 0;
    double c_inst = 0.0;

    /* Stage 0: consistent-hypothesis propagation.  A background pixel
     * whose value repeats the previous frame keeps its label; nothing
     * adapts. */
    if ((fl & ORC_FD) && s->label[p] == 0) {
        double tau = pr->tau_fd * (0.5 + Cm);
        if (near_rel((double)D, tau)) o.near |= ORC_NEAR_FD;
        if ((double)D <= tau) {
            o.stage = ORC_ST_FD;
            label = 0;
            c_inst = 1.0;
            goto finish;
        }
    }

    /* Stage 1: running Gaussian average with its own (mean, variance). */
    if (fl & ORC_RGA) {
        double tr = 0.0;
        for (int c = 0; c < 3; c++) {
            double d = I[c] - rm[c];
            double t = d * d / (lam2 * rv[c]);
            if (t > tr) tr = t;
        }
        if (near_rel(tr, 1.0)) o.near |= ORC_NEAR_RGA;
        if (tr < 1.0) {
            o.stage = ORC_ST_RGA;
            label = 0;
            if (!halt) {
                for (int c = 0; c < 3; c++) {
                    rm[c] = rm[c] + a_eff * (I[c] - rm[c]);
                    double d = I[c] - rm[c];
                    rv[c] = clampd((1.0 - a_eff) * rv[c] + a_eff * d * d,
                                   pr->var_min, pr->var_max);
                }
            }
            c_inst = wa + wb * (1.0 - dhat) + wg * (1.0 - tr);
            goto finish;
        }
    }

    /* Stage 2 with per-channel mixtures */
    if (fl & ORC_PERCHAN) {
        o.reached_gmm = 1;
        double Mhat;
        int il;
        label = stage2_perchan(pr, s, p, I, a_eff, illum_flag, &Mhat, &o.near, &il);
        o.stage = il ? ORC_ST_ILLUM : (label ? ORC_ST_FG : ORC_ST_GMM_BG);
        double qfrac;
        if (prior_nullified(pr, s, p, I, &qfrac)) {
            double den = wb + wg;
            c_inst = den > 0.0 ? (wb * (1.0 - dhat) + wg * (1.0 - Mhat)) / den : 0.0;
        } else {
            c_inst = wa * qfrac + wb * (1.0 - dhat) + wg * (1.0 - Mhat);
        }
        goto finish;
    }

    /* Stage 2: the ordered Gaussians (Eq. 2). */
    {
        o.reached_gmm = 1;
        double r[KMAX];
        int ord[KMAX];
        /* ORC_MODE1: stage 1's copy of the rank-1 mode flows back into the
         * mixture on the transition */
        if (fl & ORC_MODE1) {
            const int k1 = s->top[p];
            for (int c = 0; c < 3; c++) {
                mu[k1 * 3 + c] = rm[c];
                var[k1 * 3 + c] = rv[c];
            }
        }
        /* 1. rank key omega^2 / mean variance, descending, ties by index */
        for (int k = 0; k < K; k++) {
            double vbar = (var[k * 3 + 0] + var[k * 3 + 1] + var[k * 3 + 2]) / 3.0;
            r[k] = w[k] * w[k] / vbar;
        }
        for (int k = 0; k < K; k++) ord[k] = k;
        for (int i = 1; i < K; i++) {            /* stable insertion sort */
            int x = ord[i], j = i - 1;
            while (j >= 0 && r[ord[j]] < r[x]) { ord[j + 1] = ord[j]; j--; }
            ord[j + 1] = x;
        }
        for (int i = 0; i + 1 < K; i++) {
            double ra = r[ord[i]], rb = r[ord[i + 1]];
            double mx = ra > rb ? ra : rb;
            if (ra != rb && fabs(ra - rb) <= NEAR_REL * mx) o.near |= ORC_NEAR_RANK;
        }
        /* 2. first match in rank order: every channel within lambda sigma */
        int m = -1, mpos = -1;
        double tm = 0.0;
        for (int j = 0; j < K; j++) {
            int k = ord[j];
            double tk = 0.0;
            for (int c = 0; c < 3; c++) {
                double d = I[c] - mu[k * 3 + c];
                double t = d * d / (lam2 * var[k * 3 + c]);
                if (t > tk) tk = t;
            }
            if (near_rel(tk, 1.0)) o.near |= ORC_NEAR_MATCH;
            if (tk < 1.0) { m = k; mpos = j; tm = tk; break; }
        }
        /* 3. background iff the weight ranked before the match is <= T,
         *    decided on the state before this frame's update */
        if (m >= 0) {
            double S = 0.0;
            for (int j = 0; j < mpos; j++) S += w[ord[j]];
            if (near_rel(S, pr->T_bg)) o.near |= ORC_NEAR_BGSET;
            label = (S <= pr->T_bg) ? 0 : 1;
        } else {
            label = 1;
        }
        o.stage = label ? ORC_ST_FG : ORC_ST_GMM_BG;
        /* 4. update with rho = the effective rate */
        int tgt;
        if (m >= 0) {
            for (int k = 0; k < K; k++)
                w[k] = (1.0 - a_eff) * w[k] + (k == m ? a_eff : 0.0);
            for (int c = 0; c < 3; c++) {
                double *pm = &mu[m * 3 + c], *pv = &var[m * 3 + c];
                *pm = *pm + a_eff * (I[c] - *pm);
                double d = I[c] - *pm;
                *pv = clampd((1.0 - a_eff) * (*pv) + a_eff * d * d,
                             pr->var_min, pr->var_max);
            }
            tgt = m;
        } else {
            for (int k = 0; k < K; k++) w[k] = (1.0 - a_eff) * w[k];
            int low = ord[K - 1];
            for (int c = 0; c < 3; c++) {
                mu[low * 3 + c] = I[c];
                var[low * 3 + c] = pr->var_init;
            }
            w[low] = pr->w_init;
            tgt = low;
        }
        double sum = 0.0;
        for (int k = 0; k < K; k++) sum += w[k];
        for (int k = 0; k < K; k++) w[k] = w[k] / sum;
        /* 5. abrupt illumination change: a foreground decision is turned
         *    into background and the new or matched mode takes weight
         *    w_illum, the others sharing the rest in proportion */
        if (illum_flag && label == 1) {
            double so = 0.0;
            for (int k = 0; k < K; k++) if (k != tgt) so += w[k];
            if (so > 0.0) {
                for (int k = 0; k < K; k++)
                    if (k != tgt) w[k] = w[k] * (1.0 - pr->w_illum) / so;
                w[tgt] = pr->w_illum;
            } else {
                w[tgt] = 1.0;
            }
            label = 0;
            o.stage = ORC_ST_ILLUM;
        }
        /* 6. transition update: the background mode seeds the running
         *    average (only the active level adapts); with ORC_MODE1 the
         *    copy follows the mixture's new rank-1 mode, whatever the label */
        if (fl & ORC_MODE1) {
            int k1 = 0;
            double rb = -1.0, r2[KMAX];
            for (int k = 0; k < K; k++) {
                double vbar = (var[k * 3 + 0] + var[k * 3 + 1] + var[k * 3 + 2]) / 3.0;
                r2[k] = w[k] * w[k] / vbar;
                if (r2[k] > rb) { rb = r2[k]; k1 = k; }
            }
            for (int k = 0; k < K; k++)
                if (k != k1 && r2[k] != rb && fabs(r2[k] - rb) <= NEAR_REL * rb) o.near |= ORC_NEAR_RANK;
            s->top[p] = (uint8_t)k1;
            for (int c = 0; c < 3; c++) {
                rm[c] = mu[k1 * 3 + c];
                rv[c] = var[k1 * 3 + c];
            }
        } else if (label == 0) {
            for (int c = 0; c < 3; c++) {
                rm[c] = mu[tgt * 3 + c];
                rv[c] = var[tgt * 3 + c];
            }
        }
        /* 7. confidence terms; the prior term drops out when the value lies
         *    in no dominant mode of the prior ("prior nullified") */
        double qfrac;
        const int nullified = prior_nullified(pr, s, p, I, &qfrac);
        double Mhat = (m >= 0) ? (tm < 1.0 ? tm : 1.0) : 1.0;
        if (nullified) {
            double den = wb + wg;
            c_inst = den > 0.0 ? (wb * (1.0 - dhat) + wg * (1.0 - Mhat)) / den : 0.0;
        } else {
            c_inst = wa * qfrac + wb * (1.0 - dhat) + wg * (1.0 - Mhat);
        }
    }

finish:
    if (fl & ORC_CONF) s->conf[p] = (1.0 - pr->eta) * Cm + pr->eta * c_inst;
    for (int c = 0; c < 3; c++) J[c] = I[c];
    s->label[p] = (uint8_t)label;
    return o;
}

int orc_apply(const orc_params *pr, orc_state *s, const uint8_t *frame,
              uint8_t *mask, uint8_t *stage, uint8_t *near, orc_stats *st)
{
    if (check_params(pr) || !s || !frame || !mask) return -1;
    const int64_t P = (int64_t)pr->width * pr->height;
    /* the counter of the previous frame decides this frame's flag */
    const int flag = (pr->flags & ORC_ILLUM) &&
                     s->illum[0] * 1000 > (int64_t)pr->illum_permille * P;
    const int64_t n = s->illum[1];
    int64_t n_gmm = 0;
    int64_t n_st[6] = {0, 0, 0, 0, 0, 0};
    int64_t n0 = 0, n1 = 0, n2 = 0, n3 = 0, n4 = 0, n5 = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(+ : n_gmm, n0, n1, n2, n3, n4, n5)
#endif
    for (int64_t p = 0; p < P; p++) {
        px_out o = cascade_pixel(pr, s, p, frame + p * 3, flag, n);
        n_gmm += o.reached_gmm;
        n0 += o.stage == 0; n1 += o.stage == 1; n2 += o.stage == 2;
        n3 += o.stage == 3; n4 += o.stage == 4; n5 += o.stage == 5;
        mask[p] = s->label[p] ? 255 : 0;
        if (stage) stage[p] = (uint8_t)o.stage;
        if (near) near[p] = o.near;
    }
    n_st[0] = n0; n_st[1] = n1; n_st[2] = n2; n_st[3] = n3; n_st[4] = n4; n_st[5] = n5;
    s->illum[0] = n_gmm;
    s->illum[1] = n + 1;
    if (st) {
        for (int i = 0; i < 6; i++) st->n_stage[i] = n_st[i];
        st->n_gmm = n_gmm;
        st->illum_flag = flag;
        st->pad = 0;
    }
    return 0;
}

int orc_train(const orc_params *pr, const uint8_t *frames, int N, orc_state *s)
{
    return orc_train_near(pr, frames, N, s, NULL);
}

int orc_train_near(const orc_params *pr, const uint8_t *frames, int N, orc_state *s, uint8_t *near)
{
    if (check_params(pr) || !frames || !s || N < 2) return -1;
    const int64_t P = (int64_t)pr->width * pr->height;
    const int K = pr->K;
    int64_t g[3 * 32 + 1];
    const int R = orc_kde_weights(pr->kde_bw, g, 3 * 32 + 1);
    if (R < 0) return -1;

    /* scene prior and residue weights */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t p = 0; p < P; p++) {
        for (int c = 0; c < 3; c++)
            kde_one(frames, N, P, p, c, g, R, (1 << pr->kde_bits) - 1, s->kde + (p * 3 + c) * 256);
        residue_one(pr, frames, N, P, p, s->qa + p, s->qb + p);
    }

    /* mixture warm-up: component 0 takes the first frame with all the
     * weight; the others start empty (weight 0, mean 0, variance v_init) */
    const int perchan = (pr->flags & ORC_PERCHAN) != 0;
    for (int64_t p = 0; p < P; p++) {
        if (perchan)
            for (int c = 0; c < 3; c++)
                for (int k = 0; k < K; k++) s->wc[(p * 3 + c) * K + k] = k == 0 ? 1.0 : 0.0;
        for (int k = 0; k < K; k++) {
            s->w[p * K + k] = k == 0 ? 1.0 : 0.0;
            for (int c = 0; c < 3; c++) {
                s->mu[(p * K + k) * 3 + c] = k == 0 ? frames[p * 3 + c] : 0.0;
                s->var[(p * K + k) * 3 + c] = pr->var_init;
            }
        }
        for (int c = 0; c < 3; c++) {
            s->prev[p * 3 + c] = frames[p * 3 + c];
            s->rga_m[p * 3 + c] = frames[p * 3 + c];
            s->rga_v[p * 3 + c] = pr->var_init;
        }
        s->conf[p] = 0.5;
        s->label[p] = 0;
    }
    s->illum[0] = 0;
    s->illum[1] = 0;
    /* frames 1..N-1 run the cascade with every rejection stage and every
     * modulation off, i.e. the plain mixture at rate alpha */
    orc_params pw = *pr;
    pw.flags = perchan ? ORC_PERCHAN : 0u;
    uint8_t *mask = (uint8_t *)malloc((size_t)P);
    uint8_t *nf = near ? (uint8_t *)malloc((size_t)P) : NULL;
    if (!mask || (near && !nf)) { free(mask); free(nf); return -1; }
    if (near) memset(near, 0, (size_t)P);
    for (int t = 1; t < N; t++) {
        orc_apply(&pw, s, frames + (int64_t)t * P * 3, mask, NULL, nf, NULL);
        if (near)
            for (int64_t p = 0; p < P; p++) near[p] |= nf[p];
    }
    free(mask);
    free(nf);

    /* running average <- the top-ranked mode; C <- 0.5; the label and the
     * previous frame are those of the last training frame */
    for (int64_t p = 0; p < P; p++) {
        if (perchan) {
            /* each channel's running average starts at its own top mode */
            for (int c = 0; c < 3; c++) {
                const double *w = s->wc + (p * 3 + c) * K, *var = s->var + p * K * 3;
                int best = 0;
                double rb = -1.0, r[KMAX];
                for (int k = 0; k < K; k++) {
                    r[k] = w[k] * w[k] / var[k * 3 + c];
                    if (r[k] > rb) { rb = r[k]; best = k; }
                }
                if (near)
                    for (int k = 0; k < K; k++)
                        if (k != best && r[k] != rb && fabs(r[k] - rb) <= NEAR_REL * rb) near[p] |= ORC_NEAR_RANK;
                s->rga_m[p * 3 + c] = s->mu[(p * K + best) * 3 + c];
                s->rga_v[p * 3 + c] = s->var[(p * K + best) * 3 + c];
            }
            s->conf[p] = 0.5;
            continue;
        }
        const double *w = s->w + p * K, *var = s->var + p * K * 3;
        int best = 0;
        double rb = -1.0, r[KMAX];
        for (int k = 0; k < K; k++) {
            double vbar = (var[k * 3 + 0] + var[k * 3 + 1] + var[k * 3 + 2]) / 3.0;
            r[k] = w[k] * w[k] / vbar;
            if (r[k] > rb) { rb = r[k]; best = k; }
        }
        /* the top mode seeds the running average: a near-tie with another
         * key is a near decision too */
        if (near)
            for (int k = 0; k < K; k++)
                if (k != best && r[k] != rb && fabs(r[k] - rb) <= NEAR_REL * rb) near[p] |= ORC_NEAR_RANK;
        for (int c = 0; c < 3; c++) {
            s->rga_m[p * 3 + c] = s->mu[(p * K + best) * 3 + c];
            s->rga_v[p * 3 + c] = s->var[(p * K + best) * 3 + c];
        }
        s->top[p] = (uint8_t)best;
        s->conf[p] = 0.5;
    }
    s->illum[0] = 0;
    s->illum[1] = 0;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Textbook Stauffer-Grimson step (the comparison baseline; Eq. 2).     */
/* Written in the background-set form: order by omega^2/vbar, take the  */
/* first B components whose cumulative weight exceeds T, match the      */
/* first component in order within lambda sigma on every channel, and   */
/* call the pixel background when the match lies among those B.         */
/* ------------------------------------------------------------------ */
int orc_plain_gmm(const orc_params *pr, double *w_all, double *mu_all,
                  double *var_all, const uint8_t *frame, uint8_t *mask)
{
    if (check_params(pr) || !w_all || !mu_all || !var_all || !frame || !mask) return -1;
    const int64_t P = (int64_t)pr->width * pr->height;
    const int K = pr->K;
    const double lam2 = pr->lambda * pr->lambda;
    const double a = pr->alpha;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t p = 0; p < P; p++) {
        double *w = w_all + p * K, *mu = mu_all + p * K * 3, *var = var_all + p * K * 3;
        const uint8_t *I = frame + p * 3;
        double key[KMAX];
        int ord[KMAX], used[KMAX];
        for (int k = 0; k < K; k++) {
            key[k] = w[k] * w[k] / ((var[k * 3] + var[k * 3 + 1] + var[k * 3 + 2]) / 3.0);
            used[k] = 0;
        }
        /* selection of the largest remaining key, lowest index on ties */
        for (int j = 0; j < K; j++) {
            int best = -1;
            for (int k = 0; k < K; k++)
                if (!used[k] && (best < 0 || key[k] > key[best])) best = k;
            ord[j] = best;
            used[best] = 1;
        }
        /* background set: the first B modes in order, B the smallest count
         * whose cumulative weight exceeds T */
        int B = K;
        double cum = 0.0;
        for (int j = 0; j < K; j++) {
            cum += w[ord[j]];
            if (cum > pr->T_bg) { B = j + 1; break; }
        }
        int m = -1, mj = -1;
        for (int j = 0; j < K && m < 0; j++) {
            int k = ord[j], ok = 1;
            for (int c = 0; c < 3; c++) {
                double d = I[c] - mu[k * 3 + c];
                if (!(d * d / (lam2 * var[k * 3 + c]) < 1.0)) ok = 0;
            }
            if (ok) { m = k; mj = j; }
        }
        int fg = !(m >= 0 && mj < B);
        if (m >= 0) {
            for (int k = 0; k < K; k++) w[k] = (1.0 - a) * w[k] + (k == m ? a : 0.0);
            for (int c = 0; c < 3; c++) {
                mu[m * 3 + c] = mu[m * 3 + c] + a * (I[c] - mu[m * 3 + c]);
                double d = I[c] - mu[m * 3 + c];
                var[m * 3 + c] = clampd((1.0 - a) * var[m * 3 + c] + a * d * d,
                                        pr->var_min, pr->var_max);
            }
        } else {
            for (int k = 0; k < K; k++) w[k] = (1.0 - a) * w[k];
            int low = ord[K - 1];
            for (int c = 0; c < 3; c++) {
                mu[low * 3 + c] = I[c];
                var[low * 3 + c] = pr->var_init;
            }
            w[low] = pr->w_init;
        }
        double s = 0.0;
        for (int k = 0; k < K; k++) s += w[k];
        for (int k = 0; k < K; k++) w[k] = w[k] / s;
        mask[p] = fg ? 255 : 0;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Spatio-temporal grouping, training side (Sec. 2, "Clustering Similar */
/* Background - Spatio-Temporal Grouping", steps 1-2): replay the       */
/* mixture warm-up over the N training frames and, after each update at */
/* frames 1..N-1, record the pixel's dominant mode (largest            */
/* omega^2 / vbar, lowest index on ties): its mean variance vbar and    */
/* its weight omega.  The features are the spreads of the two series    */
/* over time, as population standard deviations, in the fixed-point    */
/* codes sd_v * 64 and sd_w * 65536 (round half up, at most 65535).    */
/* ------------------------------------------------------------------ */
int orc_group_features(const orc_params *pr, const uint8_t *frames, int N,
                       uint16_t *code_v, uint16_t *code_w)
{
    if (check_params(pr) || (pr->flags & ORC_PERCHAN) || !frames || !code_v || !code_w || N < 2) return -1;
    const int64_t P = (int64_t)pr->width * pr->height;
    const int K = pr->K;
    double *w = (double *)malloc(sizeof(double) * (size_t)(P * K));
    double *mu = (double *)malloc(sizeof(double) * (size_t)(P * K * 3));
    double *var = (double *)malloc(sizeof(double) * (size_t)(P * K * 3));
    double *sum = (double *)calloc((size_t)(P * 4), sizeof(double));   /* per pixel: sv, svv, sw, sww */
    double *ref = (double *)malloc(sizeof(double) * (size_t)(P * 2));  /* first value of each series */
    uint8_t *mask = (uint8_t *)malloc((size_t)P);
    if (!w || !mu || !var || !sum || !ref || !mask) {
        free(w); free(mu); free(var); free(sum); free(ref); free(mask);
        return -1;
    }
    /* the warm-up's start: component 0 holds the first frame with all the
     * weight, the others are empty */
    for (int64_t p = 0; p < P; p++)
        for (int k = 0; k < K; k++) {
            w[p * K + k] = k == 0 ? 1.0 : 0.0;
            for (int c = 0; c < 3; c++) {
                mu[(p * K + k) * 3 + c] = k == 0 ? frames[p * 3 + c] : 0.0;
                var[(p * K + k) * 3 + c] = pr->var_init;
            }
        }
    orc_params pw = *pr;
    pw.flags = 0u;
    for (int t = 1; t < N; t++) {
        orc_plain_gmm(&pw, w, mu, var, frames + (int64_t)t * P * 3, mask);
        for (int64_t p = 0; p < P; p++) {
            int best = 0;
            double kb = -1.0, vb = 0.0;
            for (int k = 0; k < K; k++) {
                const double *v = var + (p * K + k) * 3;
                const double vbar = (v[0] + v[1] + v[2]) / 3.0;
                const double key = w[p * K + k] * w[p * K + k] / vbar;
                if (key > kb) { kb = key; best = k; vb = vbar; }
            }
            const double om = w[p * K + best];
            if (t == 1) { ref[p * 2] = vb; ref[p * 2 + 1] = om; }
            /* sums of the series shifted by its first value (no cancellation) */
            const double dv = vb - ref[p * 2], dw = om - ref[p * 2 + 1];
            sum[p * 4 + 0] += dv;
            sum[p * 4 + 1] += dv * dv;
            sum[p * 4 + 2] += dw;
            sum[p * 4 + 3] += dw * dw;
        }
    }
    const double n = (double)(N - 1);
    for (int64_t p = 0; p < P; p++) {
        const double *s = sum + p * 4;
        double vv = s[1] / n - (s[0] / n) * (s[0] / n);
        double vw = s[3] / n - (s[2] / n) * (s[2] / n);
        const double sdv = vv > 0.0 ? sqrt(vv) : 0.0, sdw = vw > 0.0 ? sqrt(vw) : 0.0;
        const double cv = floor(sdv * 64.0 + 0.5), cw = floor(sdw * 65536.0 + 0.5);
        code_v[p] = (uint16_t)(cv > 65535.0 ? 65535.0 : cv);
        code_w[p] = (uint16_t)(cw > 65535.0 ? 65535.0 : cw);
    }
    free(w); free(mu); free(var); free(sum); free(ref); free(mask);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Spatio-temporal grouping, steps 4-6: K-means with K = 3 over the two */
/* feature codes, each feature scaled by its standard deviation over   */
/* all pixels; the cluster core of Eq. 3 (both features strictly within */
/* the cluster's mean +- its standard deviation); the core's shared     */
/* dominant mode.  Sums of the integer codes are exact; distances are  */
/* plain FP64, with a near-tie record for the assignment decision.      */
/* ------------------------------------------------------------------ */
/* Scaled distance of the codes (qv, qw) to centroid c: both features
 * divided by their spread over all pixels, squared and summed. */
static double group_dist(double qv, double qw, const double c[2], const double sd[2])
{
    const double tv = (qv - c[0]) / sd[0], tw = (qw - c[1]) / sd[1];
    return tv * tv + tw * tw;
}

/* An upper bound on how far a single-precision evaluation of group_dist
 * can land from the exact distance, when the centroid and the reciprocal
 * scales are rounded to single precision first and every operation is
 * rounded (standard model: each rounding a relative error of at most
 * u = 2^-24).  Per feature the scaled difference t is off by at most
 * delta = u (|c| + 3 |q - c|) / sd (to first order, 1 % added for the
 * second); squaring adds 2 |t| delta + delta^2; the two squares and their
 * sum add 4 u d. */
static double group_dist_fp32_err(double qv, double qw, const double c[2], const double sd[2])
{
    const double u = 1.0 / 16777216.0;
    const double dv = 1.01 * u * (fabs(c[0]) + 3.0 * fabs(qv - c[0])) / sd[0];
    const double dw = 1.01 * u * (fabs(c[1]) + 3.0 * fabs(qw - c[1])) / sd[1];
    const double tv = fabs(qv - c[0]) / sd[0], tw = fabs(qw - c[1]) / sd[1];
    return 2.0 * tv * dv + dv * dv + 2.0 * tw * dw + dw * dw + 4.0 * u * (tv * tv + tw * tw);
}

/* Nearest of the three centroids, ties to the lower cluster.  *near is set
 * when the two smallest distances lie within 1e-5 relative of each other,
 * or within twice the sum of their single-precision error bounds: a
 * single-precision implementation may legitimately pick either there. */
static int nearest3(uint16_t qv, uint16_t qw, const double c[3][2], const double sd[2], int *near)
{
    double d[3];
    int best = 0;
    for (int j = 0; j < 3; j++) {
        d[j] = group_dist(qv, qw, c[j], sd);
        if (d[j] < d[best]) best = j;
    }
    int second = best == 0 ? 1 : 0;
    for (int j = 0; j < 3; j++)
        if (j != best && d[j] < d[second]) second = j;
    const double gap = d[second] - d[best];
    const double err = group_dist_fp32_err(qv, qw, c[best], sd) + group_dist_fp32_err(qv, qw, c[second], sd);
    *near = gap <= 1e-5 * (1.0 + d[best]) || gap <= 2.0 * err;
    return best;
}

int orc_group_init(int64_t P, const uint16_t *code_v, const uint16_t *code_w, double c[3][2], double sd[2])
{
    if (P < 1 || !code_v || !code_w || !c || !sd) return -1;
    int64_t S1[2] = {0, 0}, S2[2] = {0, 0};
    for (int64_t p = 0; p < P; p++) {
        S1[0] += code_v[p];
        S1[1] += code_w[p];
        S2[0] += (int64_t)code_v[p] * code_v[p];
        S2[1] += (int64_t)code_w[p] * code_w[p];
    }
    /* sd0: the spread of a feature (0 when constant); sd: its distance
     * scale (1 when constant); first centroids on the diagonal at
     * mean - sd0, mean, mean + sd0 */
    for (int f = 0; f < 2; f++) {
        const double mean = (double)S1[f] / (double)P;
        const double v = (double)S2[f] / (double)P - mean * mean;
        const double sd0 = v > 0.0 ? sqrt(v) : 0.0;
        sd[f] = v > 0.0 ? sd0 : 1.0;
        for (int j = 0; j < 3; j++) c[j][f] = mean + (double)(j - 1) * sd0;
    }
    return 0;
}

int orc_group_centroids(int64_t P, const uint16_t *code_v, const uint16_t *code_w, const uint8_t *labels,
                        double c[3][2])
{
    if (P < 1 || !code_v || !code_w || !labels || !c) return -1;
    int64_t n[3] = {0, 0, 0}, T[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    for (int64_t p = 0; p < P; p++) {
        const int j = labels[p] & 0x7f;
        if (j > 2) return -1;
        n[j]++;
        T[j][0] += code_v[p];
        T[j][1] += code_w[p];
    }
    for (int j = 0; j < 3; j++)
        if (n[j] > 0)
            for (int f = 0; f < 2; f++) c[j][f] = (double)T[j][f] / (double)n[j];
    return 0;
}

int64_t orc_group_assign(int64_t P, const uint16_t *code_v, const uint16_t *code_w, const double c[3][2],
                         const double sd[2], uint8_t *labels, uint8_t *near)
{
    if (P < 1 || !code_v || !code_w || !c || !sd || !labels || !(sd[0] > 0.0) || !(sd[1] > 0.0)) return -1;
    int64_t n_near = 0;
    for (int64_t p = 0; p < P; p++) {
        int nr = 0;
        labels[p] = (uint8_t)nearest3(code_v[p], code_w[p], c, sd, &nr);
        if (near) near[p] = (uint8_t)nr;
        n_near += nr;
    }
    return n_near;
}

int orc_group_cluster(int64_t P, const uint16_t *code_v, const uint16_t *code_w, int max_iter,
                      uint8_t *labels, orc_group_out *out)
{
    if (P < 1 || !code_v || !code_w || !labels || !out || max_iter < 0) return -1;
    memset(out, 0, sizeof(*out));
    double c[3][2], sd[2];
    orc_group_init(P, code_v, code_w, c, sd);
    uint8_t *next = (uint8_t *)malloc((size_t)P);
    if (!next) return -1;
    out->n_near = orc_group_assign(P, code_v, code_w, c, sd, labels, NULL);
    /* Lloyd iterations: centroids <- member means (an empty cluster keeps
     * its centroid), reassign, until no label changes */
    out->iterations = max_iter;
    out->converged = 0;
    for (int it = 1; it <= max_iter; it++) {
        orc_group_centroids(P, code_v, code_w, labels, c);
        out->n_near += orc_group_assign(P, code_v, code_w, c, sd, next, NULL);
        int64_t changed = 0;
        for (int64_t p = 0; p < P; p++) {
            changed += next[p] != labels[p];
            labels[p] = next[p];
        }
        if (changed == 0) {
            out->iterations = it;
            out->converged = 1;
            break;
        }
    }
    free(next);
    return orc_group_cores(P, code_v, code_w, labels, out);
}

int orc_group_cores(int64_t P, const uint16_t *code_v, const uint16_t *code_w, uint8_t *labels, orc_group_out *out)
{
    if (P < 1 || !code_v || !code_w || !labels || !out) return -1;
    for (int j = 0; j < 3; j++) {
        out->n[j] = out->n_core[j] = 0;
        for (int f = 0; f < 2; f++) {
            out->s1[j][f] = out->s2[j][f] = 0;
            out->centroid[j][f] = out->sd[j][f] = 0.0;
        }
    }
    /* cluster statistics of the labels and the cores of Eq. 3 */
    for (int64_t p = 0; p < P; p++) {
        labels[p] &= 0x7f;
        const int j = labels[p];
        if (j > 2) return -1;
        out->n[j]++;
        out->s1[j][0] += code_v[p];
        out->s1[j][1] += code_w[p];
        out->s2[j][0] += (int64_t)code_v[p] * code_v[p];
        out->s2[j][1] += (int64_t)code_w[p] * code_w[p];
    }
    for (int j = 0; j < 3; j++)
        for (int f = 0; f < 2; f++) {
            if (out->n[j] == 0) continue;
            const double m = (double)out->s1[j][f] / (double)out->n[j];
            const double v = (double)out->s2[j][f] / (double)out->n[j] - m * m;
            out->centroid[j][f] = m;
            out->sd[j][f] = v > 0.0 ? sqrt(v) : 0.0;
        }
    for (int64_t p = 0; p < P; p++) {
        const int j = labels[p];
        const int core = fabs((double)code_v[p] - out->centroid[j][0]) < out->sd[j][0] &&
                         fabs((double)code_w[p] - out->centroid[j][1]) < out->sd[j][1];
        if (core) {
            labels[p] = (uint8_t)(j | 0x80);
            out->n_core[j]++;
        }
    }
    return 0;
}

int orc_group_params(const orc_params *pr, const orc_state *s, const uint8_t *labels, orc_group_out *out)
{
    if (check_params(pr) || (pr->flags & ORC_PERCHAN) || !s || !labels || !out) return -1;
    const int64_t P = (int64_t)pr->width * pr->height;
    const int K = pr->K;
    double acc[3][5];
    int64_t n[3] = {0, 0, 0};
    memset(acc, 0, sizeof(acc));
    for (int64_t p = 0; p < P; p++) {
        if (!(labels[p] & 0x80)) continue;
        const int j = labels[p] & 3, k = s->top[p];
        if (j > 2) return -1;
        const double *v = s->var + (p * K + k) * 3;
        acc[j][0] += s->w[p * K + k];
        for (int c = 0; c < 3; c++) acc[j][1 + c] += s->mu[(p * K + k) * 3 + c];
        acc[j][4] += (v[0] + v[1] + v[2]) / 3.0;
        n[j]++;
    }
    for (int j = 0; j < 3; j++) {
        if (!n[j]) continue;
        out->w1[j] = acc[j][0] / (double)n[j];
        for (int c = 0; c < 3; c++) out->mu1[j][c] = acc[j][1 + c] / (double)n[j];
        out->v1[j] = acc[j][4] / (double)n[j];
    }
    return 0;
}
