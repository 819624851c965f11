/*
 * FP64 CPU oracle of the Downstream tracking + two-track vertexing path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file: it is used by tests/, by __graft_entry__.smoke() (to check a
 * GPU result) and by bench.py's CPU-baseline leg.  It shares no code, header or
 * constant with the CUDA path; both read the same seeded inputs.
 *
 * It restates the method of "A Downstream and Vertexing Algorithm for Long
 * Lived Particles (LLP) Selection at the First High Level Trigger (HLT1) of
 * LHCb" (arXiv:2503.13092) step by step, in double precision, with plain loops
 * over every hit (no bucketing, no early exits, no reordering):
 *
 *   magnet point        Algorithm Design section, Eq. 1 (kink at the magnet point)
 *   UTbX window          Algorithm Design, Dv0: window opened in UTbX, up to 10
 *                        closest hits kept, seeds without hits skipped
 *   refined windows      Algorithm Design, Dv0: trajectory through the UTbX hit and
 *                        the magnet point; closest hit in UTaX, two closest in UTaU
 *                        and UTbV form candidates
 *   candidate fit/score  Algorithm Design: score from the distance between expected
 *                        and real hit positions; UT reconstructibility rule (Track
 *                        Types section)
 *   ghost killer         Ghost-Killer Neural Network section (FFNN, ReLU hidden,
 *                        sigmoid output); Ghost Rejection: keep if response < 0.5
 *   clone killing        Algorithm Design: pairs sharing more than two UT hits, the
 *                        worse one is killed
 *   vertexing            Vertexing Two Downstream Tracks, Eqs. 3-4: quadratic x(z),
 *                        Newton-Raphson point of closest approach; opposite charges
 *                        (Expected Physics Impact section)
 *
 * Where the paper is silent (window sizes, tie-breaks, fit model, the 16
 * network inputs, pick key, stopping rule) the reading taken is stated at the
 * step below.
 *
 * Every decision that could flip under a different rounding (window edges,
 * k-closest boundaries, key comparisons, thresholds) lowers a per-seed "margin":
 * margin = |a - b| / max(|a|, |b|, s), s being the magnitude of the operands.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_K1 64

typedef struct {
    /* geometry of the UT and of the kink model */
    double z[4];        /* UTaX, UTaU, UTbV, UTbX */
    double dxdy[4];     /* tan(stereo angle) */
    double z_seed;      /* z of the SciFi seed state */
    double zmag[4];     /* z_magnet = c0 + c1*tx^2 + c2*ty^2 + c3*|q/p| */
    double kappa;       /* transverse kick (MeV/c) of the kink model */
    double mp;          /* magnet polarity */
    double gamma0, gamma1; /* Eq. 3 */
    double z_ref;       /* reference plane of the track state (UT midpoint) */
    double sigma_hit, sigma_mag;
    /* method parameters */
    double w1a, w1b;    /* first window half-width: w1a + w1b*|q/p| */
    double w2;          /* refined window half-width */
    double dy_tol;      /* y tolerance on the strip extent */
    double nn_threshold;
    double doca_max;
    double nr_tol;
    int k1;             /* hits kept in UTbX (10) */
    int first_window_origin; /* 1: window centre from a line through (0,0,0) */
    int pick_chi2;      /* 1: best candidate by chi2/ndof, then ghost cut */
    int clone_kill;
    int training;       /* fixed windows 100/10 mm, clone killing off */
    int nr_max_iter;
    int variant;        /* 0: Dv0; 1: Dv1 (triplet search in UTaX x UTbX) */
    double dv1_dtx_max; /* Dv1: largest kink |tx_UT - tx_seed| a UTbX hit may imply */
    double dv1_w_tri;   /* Dv1: UTaX hit within this distance of the magnet-point line */
    double chi2_margin_scale; /* margin of a chi2 comparison per unit of relative gap */
} or_config;

typedef struct {
    int n_in, n_h1, n_h2, pad;
    const float *w1, *b1, *w2, *b2, *w3;
    const float *mean, *scale;
    float b3;
} or_nn;

/* ------------------------------------------------------------------ margins */

static void upd_margin(double *m, double a, double b, double s)
{
    double d = fabs(a - b);
    double n = fmax(fmax(fabs(a), fabs(b)), s);
    double r = n > 0.0 ? d / n : 0.0;
    if (r < *m) *m = r;
}

/* Key comparisons: a network response is compared on an absolute scale; a
 * chi2 (or chi2/ndof) comparison's relative gap is multiplied by
 * chi2_scale.  With 1e-2 the gap counts in units of the chi2 tolerance (1e-3
 * relative), so a 1e-3 relative gap maps to a margin of 1e-5. */
static void upd_key_margin(double *m, int is_chi2, double a, double b, double chi2_scale)
{
    if (is_chi2) {
        double r = fabs(a - b) / fmax(fmax(fabs(a), fabs(b)), 1e-300) * chi2_scale;
        if (r < *m) *m = r;
    } else {
        upd_margin(m, a, b, 1.0);
    }
}

/* ------------------------------------------------------------- ghost killer */

/* Ghost-Killer Neural Network section: inputs -> ReLU hidden layer(s) ->
 * output node; or_mlp applies the sigmoid.  Double precision throughout. */
double or_mlp_logit(const or_nn *nn, const double *phi)
{
    double xin[32], h1[64], h2[64];
    for (int i = 0; i < nn->n_in; ++i)
        xin[i] = (phi[i] - (double)nn->mean[i]) * (double)nn->scale[i];
    for (int o = 0; o < nn->n_h1; ++o) {
        double a = nn->b1[o];
        for (int i = 0; i < nn->n_in; ++i) a += (double)nn->w1[o * nn->n_in + i] * xin[i];
        h1[o] = a > 0.0 ? a : 0.0;
    }
    const double *last = h1;
    int n_last = nn->n_h1;
    if (nn->n_h2 > 0) {
        for (int o = 0; o < nn->n_h2; ++o) {
            double a = nn->b2[o];
            for (int i = 0; i < nn->n_h1; ++i) a += (double)nn->w2[o * nn->n_h1 + i] * h1[i];
            h2[o] = a > 0.0 ? a : 0.0;
        }
        last = h2;
        n_last = nn->n_h2;
    }
    double out = nn->b3;
    for (int i = 0; i < n_last; ++i) out += (double)nn->w3[i] * last[i];
    return out;
}

double or_mlp(const or_nn *nn, const double *phi)
{
    return 1.0 / (1.0 + exp(-or_mlp_logit(nn, phi)));
}

/* -------------------------------------------------------------- per seed */

typedef struct {
    int hit[4];            /* original hit ids, -1 = absent */
    double state[5];       /* x, y, tx, ty, q/p at z_ref */
    double chi2;
    int ndof;
    double f;              /* ghost-killer response */
    double logit;          /* network output before the sigmoid */
    double k1, k2;         /* pick key components */
    double phi[16];
} or_cand;

typedef struct {          /* one event's hits, as read from the input arrays */
    int n;
    const float *x0, *ybeg, *yend;
    const uint8_t *layer;
    int id0;               /* global id of the event's first hit */
} or_event_hits;

typedef struct { double d; int id; int idx; } or_ranked;

static int cmp_ranked(const void *a, const void *b)
{
    const or_ranked *x = (const or_ranked *)a, *y = (const or_ranked *)b;
    if (x->d < y->d) return -1;
    if (x->d > y->d) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

/* Collect hits of layer l that fall in the window |x0 - u_pred| < w and whose
 * strip extent contains y (with tolerance dy_tol); rank them by (|dx|, id) and
 * keep the closest `keep`.  Returns the number kept; out[] holds local indices. */
static int window_search(const or_config *c, const or_event_hits *ev, int l, double u_pred,
                         double y, double w, int keep, int *out, double *out_d, double *m,
                         double sx_seed, double sy_seed)
{
    or_ranked *q = (or_ranked *)malloc(sizeof(or_ranked) * (size_t)(ev->n > 0 ? ev->n : 1));
    int nq = 0;
    for (int h = 0; h < ev->n; ++h) {
        if (ev->layer[h] != l) continue;
        double x0 = ev->x0[h];
        double dx = x0 - u_pred;
        double lo = (double)ev->ybeg[h] - c->dy_tol;
        double hi = (double)ev->yend[h] + c->dy_tol;
        int in_x = fabs(dx) < w;
        int in_y = (lo <= y) && (y <= hi);
        double sx = fmax(fmax(fabs(x0), fabs(u_pred)), sx_seed);
        if (in_y) upd_margin(m, fabs(dx), w, sx);
        if (in_x) {
            upd_margin(m, y, lo, sy_seed);
            upd_margin(m, y, hi, sy_seed);
        }
        if (in_x && in_y) {
            q[nq].d = fabs(dx);
            q[nq].id = ev->id0 + h;
            q[nq].idx = h;
            ++nq;
        }
    }
    qsort(q, (size_t)nq, sizeof(or_ranked), cmp_ranked);
    if (nq > keep) upd_margin(m, q[keep - 1].d, q[keep].d, fmax(fabs(u_pred), sx_seed));
    int n = nq < keep ? nq : keep;
    for (int i = 0; i < n; ++i) {
        out[i] = q[i].idx;
        if (out_d) out_d[i] = q[i].d;
    }
    free(q);
    return n;
}

/* Lexicographic pick key: (k1, k2, hit ids in layer order, absent last). */
static int key_less(const or_cand *a, const or_cand *b)
{
    if (a->k1 != b->k1) return a->k1 < b->k1;
    if (a->k2 != b->k2) return a->k2 < b->k2;
    for (int l = 0; l < 4; ++l) {
        unsigned ua = (unsigned)a->hit[l], ub = (unsigned)b->hit[l]; /* -1 -> max */
        if (ua != ub) return ua < ub;
    }
    return 0;
}

/* Weighted straight-line least squares for x(z) = x_r + t (z - z_ref):
 * one row per present hit (measurement x0 + dxdy*y at the hit's z, weight
 * 1/sigma_hit^2) and one row for the magnet point (x_mag at z_mag, weight
 * 1/sigma_mag^2).  Solved through the 2x2 normal equations. */
static void fit_candidate(const or_config *c, const or_event_hits *ev, const int *loc,
                          double xm, double zm, const double *yl, double *xr, double *t,
                          double *chi2, int *ndof, double *res)
{
    double S0 = 0, S1 = 0, S2 = 0, Sy = 0, Szy = 0;
    double wh = 1.0 / (c->sigma_hit * c->sigma_hit);
    double wm = 1.0 / (c->sigma_mag * c->sigma_mag);
    int n = 0;
    for (int l = 0; l < 4; ++l) {
        if (loc[l] < 0) continue;
        double dz = c->z[l] - c->z_ref;
        double meas = (double)ev->x0[loc[l]] + c->dxdy[l] * yl[l];
        S0 += wh; S1 += wh * dz; S2 += wh * dz * dz; Sy += wh * meas; Szy += wh * dz * meas;
        ++n;
    }
    {
        double dz = zm - c->z_ref;
        S0 += wm; S1 += wm * dz; S2 += wm * dz * dz; Sy += wm * xm; Szy += wm * dz * xm;
    }
    double det = S0 * S2 - S1 * S1;
    *xr = (S2 * Sy - S1 * Szy) / det;
    *t = (S0 * Szy - S1 * Sy) / det;
    double x2 = 0.0;
    for (int l = 0; l < 4; ++l) {
        res[l] = 0.0;
        if (loc[l] < 0) continue;
        double meas = (double)ev->x0[loc[l]] + c->dxdy[l] * yl[l];
        double r = meas - (*xr + *t * (c->z[l] - c->z_ref));
        res[l] = r;
        x2 += wh * r * r;
    }
    {
        double r = xm - (*xr + *t * (zm - c->z_ref));
        x2 += wm * r * r;
    }
    *chi2 = x2;
    *ndof = n + 1 - 2;
}

typedef struct {
    const float *x, *y, *tx, *ty, *qop, *chi2;
} or_seeds;

/* Magnet point and first-window prediction of one seed.
 * out[0..2]  z, x, y of the magnet point: z from its parameterisation in the
 *            seed slopes and q/p, x and y by straight-line extrapolation of the
 *            SciFi state (Algorithm Design section, Eq. 1 kink model);
 * out[3]     predicted strip coordinate u = x - dxdy*y in UTbX.  KICK mode undoes
 *            the kink: tx_UT = tx_s + MP*kappa*(q/p)*sqrt(1 + tx^2 + ty^2);
 *            ORIGIN mode uses the line from (0, 0, 0) to the magnet point (Dv0);
 * out[4]     first window half-width w1a + w1b*|q/p| (100 mm in training mode);
 * out[5..8]  y at the four layers (no bending in y);
 * out[9]     refined window half-width (10 mm in training mode);
 * out[10]    tx_UT. */
void or_seed_prediction(const or_config *c, double x_s, double y_s, double tx_s, double ty_s,
                        double qop_s, double *out)
{
    const double zm = c->zmag[0] + c->zmag[1] * tx_s * tx_s + c->zmag[2] * ty_s * ty_s +
                      c->zmag[3] * fabs(qop_s);
    const double xm = x_s + tx_s * (zm - c->z_seed);
    const double ym = y_s + ty_s * (zm - c->z_seed);
    double tx_ut;
    if (c->first_window_origin)
        tx_ut = xm / zm;
    else
        tx_ut = tx_s + c->mp * c->kappa * qop_s * sqrt(1.0 + tx_s * tx_s + ty_s * ty_s);
    double yl[4];
    for (int l = 0; l < 4; ++l) yl[l] = ym + ty_s * (c->z[l] - zm);
    const double x_bx = xm + tx_ut * (c->z[3] - zm);
    out[0] = zm;
    out[1] = xm;
    out[2] = ym;
    out[3] = x_bx - c->dxdy[3] * yl[3];
    out[4] = c->training ? 100.0 : c->w1a + c->w1b * fabs(qop_s);
    for (int l = 0; l < 4; ++l) out[5 + l] = yl[l];
    out[9] = c->training ? 10.0 : c->w2;
    out[10] = tx_ut;
}

/* Dv1 (Algorithm Design section): triplets (magnet point, UTaX hit, UTbX hit)
 * in the axial layers, with no momentum-dependent first window.  Every UTbX
 * hit whose strip spans y and whose implied kink is physical,
 * |tx' - tx_s| < dtx_max with tx' = (x_h - x_m)/(z_bX - z_m) (a window of
 * half-width dtx_max (z_m - z_bX) around the straight extrapolation of the
 * seed), is joined to the magnet point; the closest UTaX hit (by (|dx|, id))
 * within w_tri of that line at z_aX completes the triplet, whose residual is
 * that distance.  Triplets are ranked by (residual, UTbX hit id) and the first
 * `keep` are kept: bx (UTbX), ax (UTaX) local indices, d (residual). */
static int triplet_search(const or_config *c, const or_event_hits *ev, double xm, double zm, double tx_s,
                          const double *yl, int keep, int *bx, int *ax, double *d, double *m, double sxs,
                          double sys)
{
    const double w_b = c->dv1_dtx_max * (zm - c->z[3]);
    const double u0 = xm + tx_s * (c->z[3] - zm) - c->dxdy[3] * yl[3];
    int *cand = (int *)malloc(sizeof(int) * (size_t)(ev->n > 0 ? ev->n : 1));
    double *cd = (double *)malloc(sizeof(double) * (size_t)(ev->n > 0 ? ev->n : 1));
    const int nb = window_search(c, ev, 3, u0, yl[3], w_b, ev->n > 0 ? ev->n : 1, cand, cd, m, sxs, sys);
    or_ranked *q = (or_ranked *)malloc(sizeof(or_ranked) * (size_t)(nb > 0 ? nb : 1));
    int *qa = (int *)malloc(sizeof(int) * (size_t)(nb > 0 ? nb : 1));
    int nq = 0;
    for (int k = 0; k < nb; ++k) {
        const int hb = cand[k];
        const double x_h = (double)ev->x0[hb] + c->dxdy[3] * yl[3];
        const double txp = (x_h - xm) / (c->z[3] - zm);
        const double ua = x_h + txp * (c->z[0] - c->z[3]) - c->dxdy[0] * yl[0];
        int a;
        double da;
        if (window_search(c, ev, 0, ua, yl[0], c->dv1_w_tri, 1, &a, &da, m, sxs, sys) == 0) continue;
        q[nq].d = da;
        q[nq].id = ev->id0 + hb;
        q[nq].idx = nq;
        qa[nq] = a;
        cand[nq] = hb;      /* compact in place: k >= nq */
        ++nq;
    }
    qsort(q, (size_t)nq, sizeof(or_ranked), cmp_ranked);
    if (nq > keep) upd_margin(m, q[keep - 1].d, q[keep].d, c->dv1_w_tri);
    const int n = nq < keep ? nq : keep;
    for (int i = 0; i < n; ++i) {
        bx[i] = cand[q[i].idx];
        ax[i] = qa[q[i].idx];
        d[i] = q[i].d;
    }
    free(q); free(qa); free(cand); free(cd);
    return n;
}

/* Full per-seed method.  Returns the number of candidates; the winner (if any)
 * goes to *best and *has_best is set.  cands/max_c optionally receive every
 * candidate (for tests and for training-sample dumps). */
static int process_seed(const or_config *c, const or_nn *nn, const or_event_hits *ev,
                        const or_seeds *sd, int s, or_cand *best, int *has_best, double *margin,
                        int *n_bx_out, or_cand *cands, int max_c)
{
    const double x_s = sd->x[s], y_s = sd->y[s], tx_s = sd->tx[s], ty_s = sd->ty[s];
    const double qop_s = sd->qop[s], chi2_s = sd->chi2[s];
    double m = INFINITY;
    double pred[11];
    or_seed_prediction(c, x_s, y_s, tx_s, ty_s, qop_s, pred);
    const double zm = pred[0], xm = pred[1], ym = pred[2], u_bx = pred[3], w1 = pred[4];
    double yl[4] = {pred[5], pred[6], pred[7], pred[8]};
    const double w2 = pred[9];
    /* magnitudes of the intermediates behind the predictions: a window or
     * strip decision is only as sharp as the largest coordinate it came from */
    const double sxs = fmax(fmax(fabs(x_s), fabs(tx_s * (zm - c->z_seed))), fmax(fabs(xm), 1.0));
    const double sys = fmax(fmax(fabs(y_s), fabs(ty_s * (zm - c->z_seed))), fmax(fabs(ym), 1.0));

    int bx[OR_MAX_K1], ax[OR_MAX_K1];
    double bx_d[OR_MAX_K1];
    const int k1 = c->k1 < OR_MAX_K1 ? c->k1 : OR_MAX_K1;
    int nbx;
    if (c->variant == 1)
        nbx = triplet_search(c, ev, xm, zm, tx_s, yl, k1, bx, ax, bx_d, &m, sxs, sys);
    else
        nbx = window_search(c, ev, 3, u_bx, yl[3], w1, k1, bx, bx_d, &m, sxs, sys);
    if (n_bx_out) *n_bx_out = nbx;

    int ncand = 0;
    int have = 0;
    or_cand win;
    memset(&win, 0, sizeof(win));
    /* keep every candidate's key to measure the winner's margin */
    or_cand *all = (or_cand *)malloc(sizeof(or_cand) * (size_t)(nbx * 4 + 1));

    for (int j = 0; j < nbx; ++j) {
        const int hb = bx[j];
        const double x_h = (double)ev->x0[hb] + c->dxdy[3] * yl[3];
        const double txp = (x_h - xm) / (c->z[3] - zm);
        int sel[3][2], nsel[3];
        const int keep[3] = {1, 2, 2};
        for (int l = 0; l < 3; ++l) {
            if (l == 0 && c->variant == 1) {   /* Dv1: the triplet's UTaX hit */
                sel[0][0] = ax[j];
                nsel[0] = 1;
                continue;
            }
            double xl = x_h + txp * (c->z[l] - c->z[3]);
            double ul = xl - c->dxdy[l] * yl[l];
            nsel[l] = window_search(c, ev, l, ul, yl[l], w2, keep[l], sel[l], NULL, &m, sxs, sys);
        }
        /* options per layer: its kept hits, or "absent" only if none qualified */
        int na = nsel[0] ? nsel[0] : 1, nu = nsel[1] ? nsel[1] : 1, nv = nsel[2] ? nsel[2] : 1;
        for (int ia = 0; ia < na; ++ia)
            for (int iu = 0; iu < nu; ++iu)
                for (int iv = 0; iv < nv; ++iv) {
                    int loc[4];
                    loc[0] = nsel[0] ? sel[0][ia] : -1;
                    loc[1] = nsel[1] ? sel[1][iu] : -1;
                    loc[2] = nsel[2] ? sel[2][iv] : -1;
                    loc[3] = hb;
                    int nh = 0;
                    for (int l = 0; l < 4; ++l) nh += loc[l] >= 0;
                    /* UT reconstructibility: >= 1 hit in station a; >= 3 hits */
                    if (nh < 3 || (loc[0] < 0 && loc[1] < 0)) continue;
                    or_cand cd;
                    memset(&cd, 0, sizeof(cd));
                    double xr, t, chi2, res[4];
                    int ndof;
                    fit_candidate(c, ev, loc, xm, zm, yl, &xr, &t, &chi2, &ndof, res);
                    double yr = ym + ty_s * (c->z_ref - zm);
                    double qop;
                    if (c->kappa != 0.0) {
                        double qopz = c->mp * (t - tx_s) / c->kappa;
                        qop = qopz / sqrt(1.0 + t * t + ty_s * ty_s);
                    } else {
                        qop = qop_s;
                    }
                    for (int l = 0; l < 4; ++l) cd.hit[l] = loc[l] >= 0 ? ev->id0 + loc[l] : -1;
                    cd.state[0] = xr; cd.state[1] = yr; cd.state[2] = t; cd.state[3] = ty_s;
                    cd.state[4] = qop;
                    cd.chi2 = chi2;
                    cd.ndof = ndof;
                    /* the 16 network inputs */
                    double *p = cd.phi;
                    p[0] = xr / 1000.0; p[1] = yr / 1000.0; p[2] = t; p[3] = ty_s;
                    p[4] = 1000.0 * qop; p[5] = chi2 / ndof;
                    p[6] = 1000.0 * qop_s; p[7] = chi2_s;
                    for (int l = 0; l < 4; ++l) p[8 + l] = res[l] / c->sigma_hit;
                    p[12] = nh / 4.0;
                    p[13] = c->variant == 1 ? bx_d[j] / c->dv1_w_tri : bx_d[j] / w1;
                    p[14] = tx_s; p[15] = ty_s;
                    /* candidates are ranked by the network output before the
                     * sigmoid: the same order as the response, without the
                     * sigmoid's saturation at 0 and 1 */
                    cd.logit = or_mlp_logit(nn, p);
                    cd.f = 1.0 / (1.0 + exp(-cd.logit));
                    if (c->pick_chi2) { cd.k1 = chi2 / ndof; cd.k2 = cd.logit; }
                    else { cd.k1 = cd.logit; cd.k2 = chi2; }
                    if (cands && ncand < max_c) cands[ncand] = cd;
                    all[ncand] = cd;
                    ++ncand;
                }
    }

    /* best pick: NN mode takes the lowest response among those under the
     * threshold; chi2 mode takes the lowest chi2/ndof and applies the cut after */
    const double T = c->nn_threshold;
    int wi = -1;
    for (int i = 0; i < ncand; ++i) {
        if (!c->pick_chi2 && !(all[i].f < T)) continue;
        if (wi < 0 || key_less(&all[i], &all[wi])) wi = i;
    }
    if (wi >= 0) {
        win = all[wi];
        /* margin against the runner-up and against the threshold */
        for (int i = 0; i < ncand; ++i) {
            if (i == wi) continue;
            int elig = c->pick_chi2 || all[i].f < T;
            if (elig) {
                if (all[i].k1 != win.k1) upd_key_margin(&m, c->pick_chi2, all[i].k1, win.k1, c->chi2_margin_scale);
                else upd_key_margin(&m, !c->pick_chi2, all[i].k2, win.k2, c->chi2_margin_scale);
            } else if (key_less(&all[i], &win)) {
                upd_margin(&m, all[i].f, T, 1.0);
            }
        }
        upd_margin(&m, win.f, T, 1.0);
        if (c->pick_chi2 && !(win.f < T)) wi = -1;
        else have = 1;
    } else {
        for (int i = 0; i < ncand; ++i) upd_margin(&m, all[i].f, T, 1.0);
    }
    free(all);
    *has_best = have;
    if (have) *best = win;
    *margin = m;
    return ncand;
}

/* Clone killing (Algorithm Design section): over one event's per-seed winners,
 * B is killed when some other winner A shares more than two UT hits with it and
 * has a lower key (k1, then k2, then seed order).  Every decision is taken
 * against the full set before killing, so the result does not depend on the
 * order of the pairs.  status: 0 no winner, 1 killed, 2 kept. */
void or_clone_kill(int n, const int *has, const int *hits, const double *k1, const double *k2,
                   int enabled, int k1_is_chi2, double chi2_scale, int *status, double *margin)
{
    for (int b = 0; b < n; ++b) {
        if (!has[b]) {
            status[b] = 0;
            continue;
        }
        int dead = 0;
        for (int a = 0; enabled && a < n; ++a) {
            if (a == b || !has[a]) continue;
            int shared = 0;
            for (int l = 0; l < 4; ++l) shared += hits[4 * a + l] >= 0 && hits[4 * a + l] == hits[4 * b + l];
            if (shared <= 2) continue;
            if (margin) {
                if (k1[a] != k1[b]) upd_key_margin(&margin[b], k1_is_chi2, k1[a], k1[b], chi2_scale);
                else upd_key_margin(&margin[b], !k1_is_chi2, k2[a], k2[b], chi2_scale);
            }
            int a_better = (k1[a] < k1[b]) || (k1[a] == k1[b] && k2[a] < k2[b]) ||
                           (k1[a] == k1[b] && k2[a] == k2[b] && a < b);
            if (a_better) dead = 1;
        }
        status[b] = dead ? 1 : 2;
    }
}

/* ------------------------------------------------------------ reconstruct */

/* Output per seed s:
 *   status[s]: 0 no track, 1 killed as a clone, 2 track kept
 *   hits[4s..4s+3], state[5s..5s+4], chi2[s], ndof[s], nn[s], ncand[s], nbx[s]
 *   margin[s]: smallest relative margin of the decisions behind the result */
void or_reconstruct(const or_config *c, const or_nn *nn, int n_events, const int *seed_off,
                    const float *sx, const float *sy, const float *stx, const float *sty,
                    const float *sqop, const float *schi2, const int *hit_off, const float *hx0,
                    const float *hybeg, const float *hyend, const uint8_t *hlayer,
                    int *status, int *hits, double *state, double *chi2, int *ndof, double *nn_out,
                    int *ncand, int *nbx, double *margin, int n_threads)
{
    or_seeds sd = {sx, sy, stx, sty, sqop, schi2};
    (void)n_threads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
#endif
    for (int e = 0; e < n_events; ++e) {
        or_event_hits ev;
        ev.n = hit_off[e + 1] - hit_off[e];
        ev.x0 = hx0 + hit_off[e];
        ev.ybeg = hybeg + hit_off[e];
        ev.yend = hyend + hit_off[e];
        ev.layer = hlayer + hit_off[e];
        ev.id0 = hit_off[e];
        const int s0 = seed_off[e], s1 = seed_off[e + 1];
        const int ns = s1 - s0;
        or_cand *win = (or_cand *)calloc((size_t)(ns > 0 ? ns : 1), sizeof(or_cand));
        int *has = (int *)calloc((size_t)(ns > 0 ? ns : 1), sizeof(int));
        for (int s = s0; s < s1; ++s) {
            int nb = 0;
            ncand[s] = process_seed(c, nn, &ev, &sd, s, &win[s - s0], &has[s - s0], &margin[s],
                                    &nb, NULL, 0);
            nbx[s] = nb;
        }
        int *st = (int *)calloc((size_t)(ns > 0 ? ns : 1), sizeof(int));
        int *wh = (int *)malloc(sizeof(int) * 4 * (size_t)(ns > 0 ? ns : 1));
        double *k1 = (double *)malloc(sizeof(double) * (size_t)(ns > 0 ? ns : 1));
        double *k2 = (double *)malloc(sizeof(double) * (size_t)(ns > 0 ? ns : 1));
        for (int b = 0; b < ns; ++b) {
            for (int l = 0; l < 4; ++l) wh[4 * b + l] = has[b] ? win[b].hit[l] : -1;
            k1[b] = win[b].k1;
            k2[b] = win[b].k2;
        }
        or_clone_kill(ns, has, wh, k1, k2, c->clone_kill && !c->training, c->pick_chi2, c->chi2_margin_scale,
                      st, margin + s0);
        for (int b = 0; b < ns; ++b) {
            int s = s0 + b;
            status[s] = st[b];
            if (!has[b]) continue;
            for (int l = 0; l < 4; ++l) hits[4 * s + l] = win[b].hit[l];
            for (int k = 0; k < 5; ++k) state[5 * s + k] = win[b].state[k];
            chi2[s] = win[b].chi2;
            ndof[s] = win[b].ndof;
            nn_out[s] = win[b].f;
        }
        free(st); free(wh); free(k1); free(k2);
        for (int s = s0; s < s1; ++s)
            if (!has[s - s0]) {
                for (int l = 0; l < 4; ++l) hits[4 * s + l] = -1;
                for (int k = 0; k < 5; ++k) state[5 * s + k] = 0.0;
                chi2[s] = 0.0; ndof[s] = 0; nn_out[s] = 0.0;
            }
        free(win);
        free(has);
    }
}

/* Every candidate of one seed (for tests and training samples).  `s` is the
 * global seed index, the event's hits are passed directly.  Returns the
 * candidate count (may exceed max_c; only max_c are written). */
int or_seed_candidates(const or_config *c, const or_nn *nn, const float *sx, const float *sy,
                       const float *stx, const float *sty, const float *sqop, const float *schi2,
                       int s, int n_hits, int id0, const float *hx0, const float *hybeg,
                       const float *hyend, const uint8_t *hlayer, int max_c, int *hits,
                       double *state, double *chi2, int *ndof, double *f, double *phi,
                       int *winner_index)
{
    or_seeds sd = {sx, sy, stx, sty, sqop, schi2};
    or_event_hits ev = {n_hits, hx0, hybeg, hyend, hlayer, id0};
    or_cand *cands = (or_cand *)malloc(sizeof(or_cand) * (size_t)(max_c > 0 ? max_c : 1));
    or_cand best;
    int has = 0, nb = 0;
    double m;
    int n = process_seed(c, nn, &ev, &sd, s, &best, &has, &m, &nb, cands, max_c);
    int w = n < max_c ? n : max_c;
    *winner_index = -1;
    for (int i = 0; i < w; ++i) {
        for (int l = 0; l < 4; ++l) hits[4 * i + l] = cands[i].hit[l];
        for (int k = 0; k < 5; ++k) state[5 * i + k] = cands[i].state[k];
        chi2[i] = cands[i].chi2;
        ndof[i] = cands[i].ndof;
        f[i] = cands[i].f;
        for (int k = 0; k < 16; ++k) phi[16 * i + k] = cands[i].phi[k];
        if (has && memcmp(cands[i].hit, best.hit, sizeof(best.hit)) == 0) *winner_index = i;
    }
    free(cands);
    return n;
}

/* --------------------------------------------------------------- vertexing */

/* Eq. 3: gamma(q/p) = -MP (gamma0 + gamma1 * q/p). */
double or_gamma(const or_config *c, double qop)
{
    return -c->mp * (c->gamma0 + c->gamma1 * qop);
}

/* Point of closest approach of two Eq. 4 trajectories
 *   T_k(z) = (x_k + tx_k u + g_k u^2, y_k + ty_k u, z),  u = z - z_ref,
 * minimising F(z1, z2) = |T_i(z1) - T_j(z2)|^2 / 2 by Newton-Raphson with the
 * exact 2x2 Hessian.  Start: the straight-line (g = 0) closest approach, or
 * z1 = z2 = z_ref when the lines are parallel to 1e-12.  Stop when both steps
 * are below nr_tol or after nr_max_iter steps.  Vertex = midpoint.
 * Returns flags: bit1 = not converged.  */
int or_poca(const or_config *c, const double *ti, const double *tj, double *z1o, double *z2o,
            double *pos, double *doca, int *iters)
{
    const double gi = or_gamma(c, ti[4]), gj = or_gamma(c, tj[4]);
    /* straight-line start */
    double Di[3] = {ti[2], ti[3], 1.0}, Dj[3] = {tj[2], tj[3], 1.0};
    double w0[3] = {ti[0] - tj[0], ti[1] - tj[1], 0.0};
    double a = Di[0] * Di[0] + Di[1] * Di[1] + Di[2] * Di[2];
    double b = Di[0] * Dj[0] + Di[1] * Dj[1] + Di[2] * Dj[2];
    double cc = Dj[0] * Dj[0] + Dj[1] * Dj[1] + Dj[2] * Dj[2];
    double d = Di[0] * w0[0] + Di[1] * w0[1] + Di[2] * w0[2];
    double e = Dj[0] * w0[0] + Dj[1] * w0[1] + Dj[2] * w0[2];
    double den = a * cc - b * b;
    double u1 = 0.0, u2 = 0.0;
    if (den > 1e-12 * a * cc) {
        u1 = (b * e - cc * d) / den;
        u2 = (a * e - b * d) / den;
    }
    int it = 0, flags = 0, conv = 0;
    for (it = 0; it < c->nr_max_iter; ++it) {
        double T1[3] = {ti[0] + ti[2] * u1 + gi * u1 * u1, ti[1] + ti[3] * u1, u1};
        double T2[3] = {tj[0] + tj[2] * u2 + gj * u2 * u2, tj[1] + tj[3] * u2, u2};
        double dd[3] = {T1[0] - T2[0], T1[1] - T2[1], T1[2] - T2[2]};
        double P1[3] = {ti[2] + 2.0 * gi * u1, ti[3], 1.0};
        double P2[3] = {tj[2] + 2.0 * gj * u2, tj[3], 1.0};
        double g1 = dd[0] * P1[0] + dd[1] * P1[1] + dd[2] * P1[2];
        double g2 = -(dd[0] * P2[0] + dd[1] * P2[1] + dd[2] * P2[2]);
        double H11 = P1[0] * P1[0] + P1[1] * P1[1] + P1[2] * P1[2] + dd[0] * 2.0 * gi;
        double H22 = P2[0] * P2[0] + P2[1] * P2[1] + P2[2] * P2[2] - dd[0] * 2.0 * gj;
        double H12 = -(P1[0] * P2[0] + P1[1] * P2[1] + P1[2] * P2[2]);
        double det = H11 * H22 - H12 * H12;
        if (!(det > 0.0)) break;
        double s1 = -(H22 * g1 - H12 * g2) / det;
        double s2 = -(H11 * g2 - H12 * g1) / det;
        u1 += s1;
        u2 += s2;
        if (fabs(s1) < c->nr_tol && fabs(s2) < c->nr_tol) {
            conv = 1;
            ++it;
            break;
        }
    }
    if (!conv) flags |= 2;
    double T1[3] = {ti[0] + ti[2] * u1 + gi * u1 * u1, ti[1] + ti[3] * u1, u1 + c->z_ref};
    double T2[3] = {tj[0] + tj[2] * u2 + gj * u2 * u2, tj[1] + tj[3] * u2, u2 + c->z_ref};
    for (int k = 0; k < 3; ++k) pos[k] = 0.5 * (T1[k] + T2[k]);
    *doca = sqrt((T1[0] - T2[0]) * (T1[0] - T2[0]) + (T1[1] - T2[1]) * (T1[1] - T2[1]) +
                 (T1[2] - T2[2]) * (T1[2] - T2[2]));
    *z1o = u1 + c->z_ref;
    *z2o = u2 + c->z_ref;
    *iters = it;
    return flags;
}

/* All opposite-charge pairs i < j of each event's tracks (tracks given in
 * output order, trk_off[E+1]); keep DOCA < doca_max.  Output in (event, i, j)
 * order; returns the number of vertices (only the first `cap` are written). */
long or_vertex(const or_config *c, int n_events, const int *trk_off, const float *x,
               const float *y, const float *tx, const float *ty, const float *qop, long cap,
               int *out_event, int *out_i, int *out_j, double *out_pos, double *out_doca,
               int *out_flags, int *out_iters, double *out_margin, long *out_pairs)
{
    long n = 0, pairs = 0;
    for (int e = 0; e < n_events; ++e) {
        for (int i = trk_off[e]; i < trk_off[e + 1]; ++i)
            for (int j = i + 1; j < trk_off[e + 1]; ++j) {
                if (!((double)qop[i] * (double)qop[j] < 0.0)) continue;
                ++pairs;
                double ti[5] = {x[i], y[i], tx[i], ty[i], qop[i]};
                double tj[5] = {x[j], y[j], tx[j], ty[j], qop[j]};
                double z1, z2, pos[3], doca;
                int it;
                int fl = or_poca(c, ti, tj, &z1, &z2, pos, &doca, &it);
                if (!(doca < c->doca_max)) continue;
                if (n < cap) {
                    out_event[n] = e;
                    out_i[n] = i;
                    out_j[n] = j;
                    for (int k = 0; k < 3; ++k) out_pos[3 * n + k] = pos[k];
                    out_doca[n] = doca;
                    out_flags[n] = fl;
                    out_iters[n] = it;
                    double m = INFINITY;
                    upd_margin(&m, doca, c->doca_max, 1.0);
                    out_margin[n] = m;
                }
                ++n;
            }
    }
    if (out_pairs) *out_pairs = pairs;
    return n;
}

/* ---------------------------------------------------- vertex-level physics */

/* Masses used for the hypotheses (MeV/c^2). */
#define OR_M_PI 139.57039
#define OR_M_P 938.27208
#define OR_M_KS 497.611
#define OR_M_LAMBDA 1115.683

/* Quantities of one two-track vertex (Expected Physics Impact section: K0S
 * and Lambda candidates from two opposite-charge downstream tracks; Fig. 18:
 * their masses once the vertex is known).  Track k = {x, y, tx, ty, q/p} at
 * z_ref; vertex = {x, y, z}.  Each daughter's momentum at the vertex has
 * magnitude 1/|q/p| and the direction of its Eq. 4 trajectory there:
 * slopes (tx + 2 gamma (z_v - z_ref), ty), gamma from Eq. 3.  Masses are the
 * plain definition M^2 = (E_1 + E_2)^2 - |p_1 + p_2|^2 under three
 * hypotheses: pi+ pi- (K0S), proton = positive track with pi- (Lambda), pi+
 * with antiproton = negative track (anti-Lambda).  Parent: P = p_1 + p_2, its
 * magnitude, transverse momentum, and the distance of closest approach of the
 * line {V + s P} to the beam line x = y = 0.
 * out: m_pipi, m_ppi, m_pip, |P|, P_T, ip, 1 - cos(opening), p_pos, p_neg,
 *      pt_pos, pt_neg.  The first track is taken as the positive one when
 * q/p > 0, else the second. */
void or_vertex_info(const or_config *c, const double *ti, const double *tj, const double *v, double *out)
{
    const double *tk[2] = {ti, tj};
    double p3[2][3], pm[2], u[2][3];
    for (int k = 0; k < 2; ++k) {
        const double g = or_gamma(c, tk[k][4]);
        const double txv = tk[k][2] + 2.0 * g * (v[2] - c->z_ref), tyv = tk[k][3];
        const double n = sqrt(1.0 + txv * txv + tyv * tyv);
        pm[k] = 1.0 / fabs(tk[k][4]);
        u[k][0] = txv / n; u[k][1] = tyv / n; u[k][2] = 1.0 / n;
        for (int a = 0; a < 3; ++a) p3[k][a] = pm[k] * u[k][a];
    }
    const int pos = ti[4] > 0.0 ? 0 : 1, neg = 1 - pos;
    double P[3];
    for (int a = 0; a < 3; ++a) P[a] = p3[0][a] + p3[1][a];
    const double P2 = P[0] * P[0] + P[1] * P[1] + P[2] * P[2];
    const double mpos[3] = {OR_M_PI, OR_M_P, OR_M_PI}, mneg[3] = {OR_M_PI, OR_M_PI, OR_M_P};
    for (int h = 0; h < 3; ++h) {
        const double e = sqrt(pm[pos] * pm[pos] + mpos[h] * mpos[h]) + sqrt(pm[neg] * pm[neg] + mneg[h] * mneg[h]);
        const double m2 = e * e - P2;
        out[h] = m2 > 0.0 ? sqrt(m2) : 0.0;
    }
    out[3] = sqrt(P2);
    const double pt = sqrt(P[0] * P[0] + P[1] * P[1]);
    out[4] = pt;
    out[5] = pt > 0.0 ? fabs(v[0] * P[1] - v[1] * P[0]) / pt : sqrt(v[0] * v[0] + v[1] * v[1]);
    out[6] = 1.0 - (u[0][0] * u[1][0] + u[0][1] * u[1][1] + u[0][2] * u[1][2]);
    out[7] = pm[pos];
    out[8] = pm[neg];
    out[9] = sqrt(p3[pos][0] * p3[pos][0] + p3[pos][1] * p3[pos][1]);
    out[10] = sqrt(p3[neg][0] * p3[neg][0] + p3[neg][1] * p3[neg][1]);
}

/* The 16 inputs of the trigger-line networks (the paper lists track, vertex
 * and parent-track parameters; this choice and its scales are the library's):
 * vertex x/100, y/100, z/1000, DOCA; |P|/1e4, P_T/1e3, ip/10;
 * (m_pipi - m_K0S)/100, (m_ppi - m_Lambda)/100, (m_pip - m_Lambda)/100;
 * p_pos/1e4, p_neg/1e4, pt_pos/1e3, pt_neg/1e3; 1e3 (1 - cos opening);
 * mean chi2/ndof of the two tracks. */
void or_line_features(const double *v, double doca, const double *info, double chi2n_i, double chi2n_j,
                      double *f)
{
    f[0] = v[0] / 100.0; f[1] = v[1] / 100.0; f[2] = v[2] / 1000.0; f[3] = doca;
    f[4] = info[3] / 1e4; f[5] = info[4] / 1e3; f[6] = info[5] / 10.0;
    f[7] = (info[0] - OR_M_KS) / 100.0;
    f[8] = (info[1] - OR_M_LAMBDA) / 100.0;
    f[9] = (info[2] - OR_M_LAMBDA) / 100.0;
    f[10] = info[7] / 1e4; f[11] = info[8] / 1e4; f[12] = info[9] / 1e3; f[13] = info[10] / 1e3;
    f[14] = 1e3 * info[6];
    f[15] = 0.5 * (chi2n_i + chi2n_j);
}

/* Every vertex of a vertexer output: info (11 per vertex), features (16) and
 * the responses of n_lines trigger-line networks (single hidden layer).
 * Track arrays in output order (chi2, ndof per track); vertices (i, j global
 * track indices, pos[3], doca). */
void or_vertex_infos(const or_config *c, long n_vtx, const int *vi, const int *vj, const double *vpos,
                     const double *vdoca, const float *x, const float *y, const float *tx, const float *ty,
                     const float *qop, const float *chi2, const int *ndof, int n_lines, const or_nn *lines,
                     double *out_info, double *out_feat, double *out_score)
{
    for (long k = 0; k < n_vtx; ++k) {
        const int i = vi[k], j = vj[k];
        double ti[5] = {x[i], y[i], tx[i], ty[i], qop[i]};
        double tj[5] = {x[j], y[j], tx[j], ty[j], qop[j]};
        double *info = out_info + 11 * k, *f = out_feat + 16 * k;
        or_vertex_info(c, ti, tj, vpos + 3 * k, info);
        const double ci = ndof[i] > 0 ? (double)chi2[i] / ndof[i] : 0.0;
        const double cj = ndof[j] > 0 ? (double)chi2[j] / ndof[j] : 0.0;
        or_line_features(vpos + 3 * k, vdoca[k], info, ci, cj, f);
        for (int l = 0; l < n_lines; ++l) out_score[n_lines * k + l] = or_mlp(&lines[l], f);
    }
}
