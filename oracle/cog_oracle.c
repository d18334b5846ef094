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
/* truncated at |d| <= 3 bw, then normalised to its peak:                */
/*   q[v] = (255 k[v] + M/2) div M,  M = max_v k[v].                      */
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
                    const int64_t *g, int R, uint8_t *q)
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
        q[v] = (uint8_t)((255 * k[v] + M / 2) / M);
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
        int qmin = 255;
        for (int c = 0; c < 3; c++) {
            int q = s->kde[(p * 3 + c) * 256 + I[c]];
            if (q < qmin) qmin = q;
        }
        if (qmin < pr->q_null) {
            double den = wb + wg;
            c_inst = den > 0.0 ? (wb * (1.0 - dhat) + wg * (1.0 - Mhat)) / den : 0.0;
        } else {
            c_inst = wa * (qmin / 255.0) + wb * (1.0 - dhat) + wg * (1.0 - Mhat);
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
        int qmin = 255;
        for (int c = 0; c < 3; c++) {
            int q = s->kde[(p * 3 + c) * 256 + I[c]];
            if (q < qmin) qmin = q;
        }
        double Mhat = (m >= 0) ? (tm < 1.0 ? tm : 1.0) : 1.0;
        if (qmin < pr->q_null) {
            double den = wb + wg;
            c_inst = den > 0.0 ? (wb * (1.0 - dhat) + wg * (1.0 - Mhat)) / den : 0.0;
        } else {
            c_inst = wa * (qmin / 255.0) + wb * (1.0 - dhat) + wg * (1.0 - Mhat);
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
            kde_one(frames, N, P, p, c, g, R, s->kde + (p * 3 + c) * 256);
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
