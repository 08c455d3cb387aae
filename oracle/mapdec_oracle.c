/*
 * FP64 CPU oracle for the BSID MAP decoder (test infrastructure only).
 *
 * This file is the plain, slow reference against which the CUDA decoder is
 * checked.  Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load it; the decoder library never does.  It shares no
 * code, header, table or helper with the CUDA path.
 *
 * Everything follows the paper's Sec. II (Preliminaries) in its own order and
 * notation, in double precision:
 *   - receiver metric R(y|x): the lattice of eqs. (F), (F_lastrow) with its
 *     initial conditions, plus a cap of I insertions per transmitted bit;
 *   - gamma_i(m', m, D) = Pr{D_i = D} R(Y[n i + m' .. n(i+1) + m) | C_i(D)),
 *     eq. (gamma), evaluated on the paper's own (i, m', D) grid, with one
 *     codebook for every symbol or a codebook C_i per symbol (the constituent
 *     encodings of Sec. II-A);
 *   - the forward recursion with per-index normalisation, eqs. (alpha),
 *     (alpha_norm), (alpha_prenorm); the backward recursion eq. (beta),
 *     normalised the same way;
 *   - the APPs, eqs. (L), (lambda), (sigma), normalised over D per symbol,
 *     and the extrinsic outputs (the same sums without the symbol's own
 *     prior), which an outer decoder takes in iterative decoding (Sec. II-A);
 *   - the frame log-likelihood  log P(Y) = sum_i log c_i + log alpha_N(rho-tau)
 *     where c_i are the forward normalisers of eq. (alpha_norm).
 *
 * Readings taken where the paper is silent (each also used by the tests):
 *   - insertions before a transmitted bit are capped at I; weights are not
 *     renormalised, so truncated paths are simply dropped;
 *   - lattice rows/columns are 1-based: row r has consumed r bits, column j
 *     has consumed j received bits; the diagonal into (r, j) compares x_r, y_j;
 *   - each inserted bit has weight Pi/2 (uniform value, never substituted);
 *   - an isolated frame with known length: alpha_0 = [m = 0],
 *     beta_N = [m = rho - tau];
 *   - drift limits: m in [-xmax, xmax] at symbol boundaries, drift change
 *     m - m' in [-n, n I]; a window that starts before 0 or runs past rho
 *     contributes nothing;
 *   - beta is normalised by its own sum; APPs are normalised over D.
 *
 * Gradients (not in the paper): d logP / d(Pi, Pd, Ps) with Pt = 1 - Pi - Pd,
 * by forward-mode dual numbers carried through every step above; and
 * d logP / d Pr{D_i = D}, which follows from P(Y) being linear in each prior:
 * P(Y) = sum_D Pr{D_i = D} Q_i(D), Q_i(D) = sum_{m',m} alpha_i(m') R beta_{i+1}(m).
 *
 * The optional memo caches R(.|C(D)) per (rx start p, D): the same lattice
 * function evaluated once per key, so results are bitwise identical to the
 * un-memoised (i, m', D) grid; it only saves time on large frames.  With
 * per-symbol codebooks the lattice at (p, D) also depends on i, and the memo
 * is off.
 *
 * Optional received-bit weight kappa (default 1: the literal recursion).  The
 * normalised forward row alpha_i(m) is the probability of a received prefix of
 * n i + m bits, so its entries fall off by roughly 2^-h per bit of drift (h the
 * entropy rate of the received bits).  On long frames with wide drift limits
 * the entries that carry the posterior fall below even the FP64 range and the
 * literal recursion reports a zero-probability frame.  With kappa != 1 every
 * gamma is multiplied by kappa^(received length), which multiplies every path
 * of the frame by the same kappa^rho: APPs are unchanged, log P(Y) is recovered
 * by subtracting rho log kappa, and the rows stay representable.  The tests
 * check that results agree with kappa = 1 wherever the literal recursion works.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_DRIFT_RANGE 2
#define ORC_ERR_ZERO_PROB 3
#define ORC_ERR_NOMEM 4

/* ------------------------------------------------------------------ */
/* Receiver metric lattice, eqs. (F), (F_lastrow), with insertion cap I */
/* ------------------------------------------------------------------ */

/*
 * x[0..n): transmitted bits x_1..x_n; y[0..mu): received bits y_1..y_mu.
 * Writes out[j] = F_{n,j}, j = 0..mu: the probability that x is received as
 * exactly y_1..y_j (eq. F_lastrow gives the last row).  The horizontal
 * (insertion, weight Pi/2) steps of eq. (F) happen in rows r < n only, at
 * most I of them in each row.  The corridor of Sec. II-C keeps only nodes
 * with j - r in [m_n^-, m_n^+] = [-n, n I].
 */
int orc_receiver_metric(int n, int I, const uint8_t *x, const uint8_t *y, int mu,
                        double Pi, double Pd, double Ps, double *out)
{
    if (n < 1 || I < 0 || mu < 0 || !x || (mu > 0 && !y) || !out) return ORC_ERR_ARG;
    const double Pt = 1.0 - Pi - Pd;
    const double half_pi = 0.5 * Pi;
    double *F = (double *)calloc((size_t)(mu + 1), sizeof(double));
    double *G = (double *)calloc((size_t)(mu + 1), sizeof(double));
    double *wp = (double *)calloc((size_t)(I + 1), sizeof(double));
    if (!F || !G || !wp) { free(F); free(G); free(wp); return ORC_ERR_NOMEM; }
    wp[0] = 1.0;
    for (int a = 1; a <= I; ++a) wp[a] = wp[a - 1] * half_pi;

    /* initial condition: F_{0,0} = 1, everything else 0 */
    F[0] = 1.0;
    for (int r = 0; r < n; ++r) {
        /* row r including its horizontal steps:
           G_{r,j} = sum_{a=0}^{min(I,j)} (Pi/2)^a F_{r,j-a}              */
        for (int j = 0; j <= mu; ++j) {
            double g = 0.0;
            for (int a = 0; a <= I && a <= j; ++a) g += wp[a] * F[j - a];
            if (j - r < -n || j - r > n * I) g = 0.0; /* corridor */
            G[j] = g;
        }
        /* row r+1 by vertical (deletion) and diagonal (transmission) steps:
           F_{r+1,j} = Pd G_{r,j} + Qdot(y_j | x_{r+1}) G_{r,j-1}             */
        for (int j = 0; j <= mu; ++j) {
            double f = Pd * G[j];
            if (j >= 1) {
                const double Q = (y[j - 1] != x[r]) ? Pt * Ps : Pt * (1.0 - Ps);
                f += Q * G[j - 1];
            }
            if (j - (r + 1) < -n || j - (r + 1) > n * I) f = 0.0; /* corridor */
            F[j] = f;
        }
    }
    memcpy(out, F, (size_t)(mu + 1) * sizeof(double));
    free(F); free(G); free(wp);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Dual numbers for forward-mode derivatives w.r.t. (Pi, Pd, Ps)       */
/* ------------------------------------------------------------------ */

typedef struct { double v, d[3]; } dual;

static inline dual d_const(double v) { dual r = {v, {0, 0, 0}}; return r; }
static inline dual d_add(dual a, dual b)
{
    dual r = {a.v + b.v, {a.d[0] + b.d[0], a.d[1] + b.d[1], a.d[2] + b.d[2]}};
    return r;
}
static inline dual d_mul(dual a, dual b)
{
    dual r;
    r.v = a.v * b.v;
    for (int k = 0; k < 3; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
static inline dual d_scale(dual a, double s)
{
    dual r = {a.v * s, {a.d[0] * s, a.d[1] * s, a.d[2] * s}};
    return r;
}
static inline dual d_div(dual a, dual b)
{
    dual r;
    r.v = a.v / b.v;
    for (int k = 0; k < 3; ++k) r.d[k] = (a.d[k] * b.v - a.v * b.d[k]) / (b.v * b.v);
    return r;
}
static inline dual d_log(dual a)
{
    dual r;
    r.v = log(a.v);
    for (int k = 0; k < 3; ++k) r.d[k] = a.d[k] / a.v;
    return r;
}

/* The same lattice as orc_receiver_metric, carried in dual numbers. */
static int orc_receiver_metric_dual(int n, int I, const uint8_t *x, const uint8_t *y, int mu,
                                    double Pi, double Pd, double Ps, dual *out)
{
    dual dPi = {Pi, {1, 0, 0}};
    dual dPd = {Pd, {0, 1, 0}};
    dual dPs = {Ps, {0, 0, 1}};
    dual dPt = d_add(d_const(1.0), d_add(d_scale(dPi, -1.0), d_scale(dPd, -1.0)));
    dual Qdiff = d_mul(dPt, dPs);
    dual Qsame = d_mul(dPt, d_add(d_const(1.0), d_scale(dPs, -1.0)));
    dual half_pi = d_scale(dPi, 0.5);
    dual *F = (dual *)calloc((size_t)(mu + 1), sizeof(dual));
    dual *G = (dual *)calloc((size_t)(mu + 1), sizeof(dual));
    dual *wp = (dual *)calloc((size_t)(I + 1), sizeof(dual));
    if (!F || !G || !wp) { free(F); free(G); free(wp); return ORC_ERR_NOMEM; }
    wp[0] = d_const(1.0);
    for (int a = 1; a <= I; ++a) wp[a] = d_mul(wp[a - 1], half_pi);
    F[0] = d_const(1.0);
    for (int r = 0; r < n; ++r) {
        for (int j = 0; j <= mu; ++j) {
            dual g = d_const(0.0);
            for (int a = 0; a <= I && a <= j; ++a) g = d_add(g, d_mul(wp[a], F[j - a]));
            if (j - r < -n || j - r > n * I) g = d_const(0.0);
            G[j] = g;
        }
        for (int j = 0; j <= mu; ++j) {
            dual f = d_mul(dPd, G[j]);
            if (j >= 1) {
                const dual Q = (y[j - 1] != x[r]) ? Qdiff : Qsame;
                f = d_add(f, d_mul(Q, G[j - 1]));
            }
            if (j - (r + 1) < -n || j - (r + 1) > n * I) f = d_const(0.0);
            F[j] = f;
        }
    }
    memcpy(out, F, (size_t)(mu + 1) * sizeof(dual));
    free(F); free(G); free(wp);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Frame context                                                       */
/* ------------------------------------------------------------------ */

static double g_kappa = 1.0;

/* Received-bit weight used by the decode entry points (1 = literal). */
void orc_set_received_bit_weight(double kappa) { g_kappa = (kappa > 0.0) ? kappa : 1.0; }

typedef struct {
    int q, n, N, I, xmax, M, Mn;
    int64_t rho;
    double Pi, Pd, Ps;
    const uint8_t *cb;  /* q*n codeword bits, or N*q*n with per-symbol codebooks */
    size_t cb_stride;   /* 0: C_i = C for every i; q*n: codebook C_i at cb + i*q*n */
    const uint8_t *rx;  /* rho received bits */
    const double *pri;  /* N*q priors, or NULL for uniform 1/q */
    const double *phi0; /* M: prior of the drift at the frame start (alpha_0), or NULL: [m = 0] */
    const double *phiN; /* M: prior of the drift at the frame end (beta_N), or NULL: [m = rho - tau] */
    int memo;
    double *Rm;         /* memo, (rho+1)*q*Mn, valid where Rk[p] set */
    uint8_t *Rk;
    dual *Rd;           /* dual memo for gradients */
    uint8_t *Rdk;
} orc_ctx;

static double orc_prior(const orc_ctx *c, int i, int D)
{
    return c->pri ? c->pri[(size_t)i * c->q + D] : 1.0 / (double)c->q;
}

/* Codeword C_i(D) of the constituent encoding of symbol i (Sec. II-A). */
static const uint8_t *orc_codeword(const orc_ctx *c, int i, int D)
{
    return c->cb + (size_t)i * c->cb_stride + (size_t)D * c->n;
}

/* R(Y[p .. p+j) | C_i(D)) for j = 0..Mn-1 (entries with p + j > rho are 0).
   The memo (keyed by p, D) is only used with one codebook for all symbols. */
static int orc_R(orc_ctx *c, int i, int64_t p, int D, double *Rj)
{
    const int Mn = c->Mn;
    if (c->memo && c->Rk[p]) {
        memcpy(Rj, c->Rm + ((size_t)p * c->q + D) * Mn, (size_t)Mn * sizeof(double));
        return ORC_OK;
    }
    int64_t avail = c->rho - p;
    int mu = (int)(avail < (int64_t)(Mn - 1) ? avail : (int64_t)(Mn - 1));
    for (int j = 0; j < Mn; ++j) Rj[j] = 0.0;
    int st = orc_receiver_metric(c->n, c->I, orc_codeword(c, i, D), c->rx + p, mu,
                                 c->Pi, c->Pd, c->Ps, Rj);
    if (st) return st;
    if (c->memo) {
        memcpy(c->Rm + ((size_t)p * c->q + D) * Mn, Rj, (size_t)Mn * sizeof(double));
        if (D == c->q - 1) c->Rk[p] = 1;
    }
    return ORC_OK;
}

static int orc_R_dual(orc_ctx *c, int i, int64_t p, int D, dual *Rj)
{
    const int Mn = c->Mn;
    if (c->memo && c->Rdk[p]) {
        memcpy(Rj, c->Rd + ((size_t)p * c->q + D) * Mn, (size_t)Mn * sizeof(dual));
        return ORC_OK;
    }
    int64_t avail = c->rho - p;
    int mu = (int)(avail < (int64_t)(Mn - 1) ? avail : (int64_t)(Mn - 1));
    for (int j = 0; j < Mn; ++j) Rj[j] = d_const(0.0);
    int st = orc_receiver_metric_dual(c->n, c->I, orc_codeword(c, i, D), c->rx + p, mu,
                                      c->Pi, c->Pd, c->Ps, Rj);
    if (st) return st;
    if (c->memo) {
        memcpy(c->Rd + ((size_t)p * c->q + D) * Mn, Rj, (size_t)Mn * sizeof(dual));
        if (D == c->q - 1) c->Rdk[p] = 1;
    }
    return ORC_OK;
}

/*
 * gamma_i(m', m, D), eq. (gamma), for all m' in [-xmax, xmax], D, and
 * drift change delta = m - m' in [-n, nI]; stored as
 * g[((m'+xmax) * q + D) * Mn + (delta + n)].  Zero where m is outside the
 * drift limits or the received window leaves [0, rho).
 * If R is non-NULL the receiver metric without the prior is stored alongside.
 */
static int orc_gamma(orc_ctx *c, int i, double *g, double *R)
{
    const int M = c->M, q = c->q, n = c->n, Mn = c->Mn, xmax = c->xmax;
    double *Rj = (double *)malloc((size_t)Mn * sizeof(double));
    if (!Rj) return ORC_ERR_NOMEM;
    for (int mp = 0; mp < M; ++mp) {
        const int m1 = mp - xmax;
        const int64_t p = (int64_t)n * i + m1;
        for (int D = 0; D < q; ++D) {
            double *gd = g + ((size_t)mp * q + D) * Mn;
            double *Rd = R ? R + ((size_t)mp * q + D) * Mn : NULL;
            if (p < 0 || p > c->rho) {
                for (int k = 0; k < Mn; ++k) { gd[k] = 0.0; if (Rd) Rd[k] = 0.0; }
                continue;
            }
            int st = orc_R(c, i, p, D, Rj);
            if (st) { free(Rj); return st; }
            const double pr = orc_prior(c, i, D);
            double kw = 1.0;  /* kappa^k, k = received length */
            for (int k = 0; k < Mn; ++k) {
                const int m2 = m1 + (k - n);
                const int inside = (m2 >= -xmax && m2 <= xmax);
                gd[k] = inside ? pr * Rj[k] * kw : 0.0;
                if (Rd) Rd[k] = inside ? Rj[k] * kw : 0.0;
                kw *= g_kappa;
            }
        }
    }
    free(Rj);
    return ORC_OK;
}

static int orc_gamma_dual(orc_ctx *c, int i, dual *g)
{
    const int M = c->M, q = c->q, n = c->n, Mn = c->Mn, xmax = c->xmax;
    dual *Rj = (dual *)malloc((size_t)Mn * sizeof(dual));
    if (!Rj) return ORC_ERR_NOMEM;
    for (int mp = 0; mp < M; ++mp) {
        const int m1 = mp - xmax;
        const int64_t p = (int64_t)n * i + m1;
        for (int D = 0; D < q; ++D) {
            dual *gd = g + ((size_t)mp * q + D) * Mn;
            if (p < 0 || p > c->rho) {
                for (int k = 0; k < Mn; ++k) gd[k] = d_const(0.0);
                continue;
            }
            int st = orc_R_dual(c, i, p, D, Rj);
            if (st) { free(Rj); return st; }
            const double pr = orc_prior(c, i, D);
            double kw = 1.0;
            for (int k = 0; k < Mn; ++k) {
                const int m2 = m1 + (k - n);
                gd[k] = (m2 >= -xmax && m2 <= xmax) ? d_scale(Rj[k], pr * kw) : d_const(0.0);
                kw *= g_kappa;
            }
        }
    }
    free(Rj);
    return ORC_OK;
}

static int orc_init(orc_ctx *c, int q, int n, const uint8_t *codebook, int per_symbol, int N,
                    double Pi, double Pd, double Ps, int I, int xmax, const uint8_t *rx,
                    int64_t rho, const double *priors, int memo, int want_dual)
{
    memset(c, 0, sizeof(*c));
    if (q < 2 || n < 1 || n > 62 || N < 1 || I < 1 || xmax < 0 || !codebook || rho < 0 ||
        (rho > 0 && !rx))
        return ORC_ERR_ARG;
    if (n < 31 && q > (1 << n)) return ORC_ERR_ARG;
    if (!(Pi >= 0 && Pd >= 0 && Ps >= 0 && Ps <= 1 && Pi + Pd < 1)) return ORC_ERR_ARG;
    int64_t tau = (int64_t)n * N;
    if (rho - tau > xmax || tau - rho > xmax) return ORC_ERR_DRIFT_RANGE;
    c->q = q; c->n = n; c->N = N; c->I = I; c->xmax = xmax;
    c->M = 2 * xmax + 1; c->Mn = n * (I + 1) + 1;
    c->rho = rho; c->Pi = Pi; c->Pd = Pd; c->Ps = Ps;
    c->cb = codebook; c->rx = rx; c->pri = priors;
    c->cb_stride = per_symbol ? (size_t)q * n : 0;
    /* with per-symbol codebooks the lattice at (p, D) depends on i as well */
    c->memo = per_symbol ? 0 : memo;
    memo = c->memo;
    if (memo) {
        size_t cells = (size_t)(rho + 1) * q * c->Mn;
        if (want_dual) {
            c->Rd = (dual *)malloc(cells * sizeof(dual));
            c->Rdk = (uint8_t *)calloc((size_t)(rho + 1), 1);
            if (!c->Rd || !c->Rdk) return ORC_ERR_NOMEM;
        }
        c->Rm = (double *)malloc(cells * sizeof(double));
        c->Rk = (uint8_t *)calloc((size_t)(rho + 1), 1);
        if (!c->Rm || !c->Rk) return ORC_ERR_NOMEM;
    }
    return ORC_OK;
}

static void orc_free(orc_ctx *c)
{
    free(c->Rm); free(c->Rk); free(c->Rd); free(c->Rdk);
    c->Rm = NULL; c->Rk = NULL; c->Rd = NULL; c->Rdk = NULL;
}

/*
 * Frame boundaries (Sec. II-C: alpha_0 and beta_N are the prior probabilities
 * of the frame boundaries).  An isolated frame has alpha_0(m) = [m = 0] and
 * beta_N(m) = [m = rho - tau].  In stream decoding the boundaries are
 * uncertain and carry drift priors phi0, phiN: the frame starts at received
 * position m0 with probability phi0(m0) (bits before it belong to the previous
 * frame) and ends at tau + mN with probability phiN(mN) (bits after it belong
 * to the next one), so
 *   P(Y) = sum_{m0, mN} phi0(m0) P(Y[m0 .. tau + mN) | frame) phiN(mN).
 * With the received-bit weight kappa every gamma carries kappa^{received
 * length}; a path from m0 to mN then carries kappa^{tau + mN - m0}.  The start
 * row is weighted kappa^{m0} and the end row kappa^{-(tau + mN)}, so every
 * path's weight cancels exactly (kappa = 1 is the paper's recursion).
 * orc_start_row writes the normalised alpha_0 and adds the log of its sum to
 * *ls; orc_end_row writes beta_N (unnormalised weights); orc_end_logp returns
 * log of sum_m alpha_N(m) beta_N(m) for the normalised alpha_N.
 */
static int orc_start_row(const orc_ctx *c, double *A, double *ls)
{
    const int M = c->M;
    if (!c->phi0) {
        for (int m = 0; m < M; ++m) A[m] = 0.0;
        A[c->xmax] = 1.0;
        return ORC_OK;
    }
    double s = 0.0;
    for (int m = 0; m < M; ++m) {
        const double v = c->phi0[m];
        if (!(v >= 0.0)) return ORC_ERR_ARG;
        A[m] = v * pow(g_kappa, (double)(m - c->xmax));
        s += A[m];
    }
    if (!(s > 0.0)) return ORC_ERR_ZERO_PROB;
    for (int m = 0; m < M; ++m) A[m] /= s;
    *ls += log(s);
    return ORC_OK;
}

/* beta_N(m) kappa^tau: the end row's weights without the common kappa^{-tau},
 * which log P takes separately (it would underflow). */
static int orc_end_row(const orc_ctx *c, double *bN)
{
    const int M = c->M;
    const int64_t tau = (int64_t)c->n * c->N;
    for (int m = 0; m < M; ++m) bN[m] = 0.0;
    if (!c->phiN) {
        bN[(int)(c->rho - tau) + c->xmax] = pow(g_kappa, -(double)(c->rho - tau));
        return ORC_OK;
    }
    for (int m = 0; m < M; ++m) {
        const double v = c->phiN[m];
        if (!(v >= 0.0)) return ORC_ERR_ARG;
        bN[m] = v * pow(g_kappa, -(double)(m - c->xmax));
    }
    return ORC_OK;
}

/* log sum_m alpha_N(m) beta_N(m), the end of log P (with -tau log kappa). */
static double orc_end_logp(const orc_ctx *c, const double *aN, const double *bN)
{
    double s = 0.0;
    for (int m = 0; m < c->M; ++m) s += aN[m] * bN[m];
    return (s > 0.0 ? log(s) : -INFINITY) - (double)((int64_t)c->n * c->N) * log(g_kappa);
}

/*
 * Forward pass, eqs. (alpha_prenorm), (alpha_norm):
 *   alpha'_{i+1}(m) = sum_{m', D} alpha_i(m') gamma_i(m', m, D),
 *   c_{i+1} = sum_m alpha'_{i+1}(m),  alpha_{i+1} = alpha'_{i+1} / c_{i+1}.
 * alpha rows (N+1)*M are written to A; returns sum_i log c_i in *logsum.
 */
static int orc_forward(orc_ctx *c, double *A, double *logsum)
{
    const int M = c->M, q = c->q, Mn = c->Mn, n = c->n;
    double *g = (double *)malloc((size_t)M * q * Mn * sizeof(double));
    if (!g) return ORC_ERR_NOMEM;
    double ls = 0.0;
    int st0 = orc_start_row(c, A, &ls);
    if (st0) { free(g); return st0; }
    for (int i = 0; i < c->N; ++i) {
        int st = orc_gamma(c, i, g, NULL);
        if (st) { free(g); return st; }
        const double *a = A + (size_t)i * M;
        double *an = A + (size_t)(i + 1) * M;
        for (int m = 0; m < M; ++m) an[m] = 0.0;
        for (int mp = 0; mp < M; ++mp)
            for (int D = 0; D < q; ++D) {
                const double *gd = g + ((size_t)mp * q + D) * Mn;
                for (int k = 0; k < Mn; ++k) {
                    const int m = mp + k - n;
                    if (m >= 0 && m < M) an[m] += a[mp] * gd[k];
                }
            }
        double cs = 0.0;
        for (int m = 0; m < M; ++m) cs += an[m];
        if (!(cs > 0.0)) { free(g); return ORC_ERR_ZERO_PROB; }
        for (int m = 0; m < M; ++m) an[m] /= cs;
        ls += log(cs);
    }
    free(g);
    *logsum = ls;
    return ORC_OK;
}

/*
 * Backward pass, eq. (beta):
 *   beta_i(m) = sum_{m', D} beta_{i+1}(m') gamma_i(m, m', D),
 * normalised by its own sum; beta_N(m) = [m = rho - tau].
 */
static int orc_backward(orc_ctx *c, double *B)
{
    const int M = c->M, q = c->q, Mn = c->Mn, n = c->n, N = c->N;
    double *g = (double *)malloc((size_t)M * q * Mn * sizeof(double));
    if (!g) return ORC_ERR_NOMEM;
    double *bN = B + (size_t)N * M;
    int st0 = orc_end_row(c, bN);
    if (st0) { free(g); return st0; }
    {  /* normalised like every other row (its scale never enters log P) */
        double ds = 0.0;
        for (int m = 0; m < M; ++m) ds += bN[m];
        if (!(ds > 0.0)) { free(g); return ORC_ERR_ZERO_PROB; }
        for (int m = 0; m < M; ++m) bN[m] /= ds;
    }
    for (int i = N - 1; i >= 0; --i) {
        int st = orc_gamma(c, i, g, NULL);
        if (st) { free(g); return st; }
        const double *bn = B + (size_t)(i + 1) * M;
        double *b = B + (size_t)i * M;
        for (int m = 0; m < M; ++m) {
            double s = 0.0;
            for (int D = 0; D < q; ++D) {
                const double *gd = g + ((size_t)m * q + D) * Mn;
                for (int k = 0; k < Mn; ++k) {
                    const int m2 = m + k - n;
                    if (m2 >= 0 && m2 < M) s += bn[m2] * gd[k];
                }
            }
            b[m] = s;
        }
        double ds = 0.0;
        for (int m = 0; m < M; ++m) ds += b[m];
        if (!(ds > 0.0)) { free(g); return ORC_ERR_ZERO_PROB; }
        for (int m = 0; m < M; ++m) b[m] /= ds;
    }
    free(g);
    return ORC_OK;
}

/*
 * APPs, eqs. (L), (sigma): L_i(D) proportional to
 *   sum_{m', m} alpha_i(m') gamma_i(m', m, D) beta_{i+1}(m),
 * normalised over D.  If Qout is given, also writes
 *   Q_i(D) = sum_{m', m} alpha_i(m') R beta_{i+1}(m)   (gamma without prior)
 * and Z_i = sum_D Pr{D_i=D} Q_i(D) to Zout.
 */
static int orc_app(orc_ctx *c, const double *A, const double *B, double *app, double *Qout,
                   double *Zout)
{
    const int M = c->M, q = c->q, Mn = c->Mn, n = c->n, N = c->N;
    double *g = (double *)malloc((size_t)M * q * Mn * sizeof(double));
    double *R = Qout ? (double *)malloc((size_t)M * q * Mn * sizeof(double)) : NULL;
    double *L = (double *)malloc((size_t)q * sizeof(double));
    if (!g || !L || (Qout && !R)) { free(g); free(R); free(L); return ORC_ERR_NOMEM; }
    for (int i = 0; i < N; ++i) {
        int st = orc_gamma(c, i, g, R);
        if (st) { free(g); free(R); free(L); return st; }
        const double *a = A + (size_t)i * M;
        const double *bn = B + (size_t)(i + 1) * M;
        double tot = 0.0;
        for (int D = 0; D < q; ++D) {
            double s = 0.0, sq = 0.0;
            for (int mp = 0; mp < M; ++mp) {
                const double *gd = g + ((size_t)mp * q + D) * Mn;
                const double *Rd = R ? R + ((size_t)mp * q + D) * Mn : NULL;
                for (int k = 0; k < Mn; ++k) {
                    const int m = mp + k - n;
                    if (m >= 0 && m < M) {
                        s += a[mp] * gd[k] * bn[m];
                        if (Rd) sq += a[mp] * Rd[k] * bn[m];
                    }
                }
            }
            L[D] = s;
            tot += s;
            if (Qout) Qout[(size_t)i * q + D] = sq;
        }
        if (!(tot > 0.0)) { free(g); free(R); free(L); return ORC_ERR_ZERO_PROB; }
        if (app)
            for (int D = 0; D < q; ++D) app[(size_t)i * q + D] = L[D] / tot;
        if (Zout) Zout[i] = tot;
    }
    free(g); free(R); free(L);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Public entry points                                                 */
/* ------------------------------------------------------------------ */

/*
 * Full decode of one frame under the constituent encodings of Sec. II-A.
 * codebooks: per_symbol = 0, one codebook C (q*n bits) used for every symbol;
 * per_symbol = 1, the codebooks C_0..C_{N-1} (N*q*n bits, C_i at i*q*n).
 * Outputs, each optional (NULL):
 *   app    N*q APPs of eq. (L), row i normalised over D;
 *   ext    N*q extrinsic outputs: E_i(D) proportional to
 *          sum_{m', m} alpha_i(m') R(Y[n i + m' .. n(i+1) + m) | C_i(D)) beta_{i+1}(m),
 *          i.e. eq. (L) without the symbol's own prior Pr{D_i = D}, row i
 *          normalised over D.  This is what the inner decoder hands to an
 *          outer decoder when the two are decoded iteratively (Sec. II-A, and
 *          the role of the priors in Sec. II-C);
 *   loglik log P(Y).
 * priors: N*q, row i = Pr{D_i = .}; NULL means uniform 1/q.
 */
int orc_decode_general(int q, int n, const uint8_t *codebooks, int per_symbol, int N, double Pi,
                       double Pd, double Ps, int I, int xmax, const uint8_t *rx, int64_t rho,
                       const double *priors, int memo, double *app, double *ext,
                       double *loglik, const double *phi0, const double *phiN)
{
    orc_ctx c;
    int st = orc_init(&c, q, n, codebooks, per_symbol, N, Pi, Pd, Ps, I, xmax, rx, rho, priors,
                      memo, 0);
    if (st) { orc_free(&c); return st; }
    c.phi0 = phi0;
    c.phiN = phiN;
    const size_t rows = (size_t)(N + 1) * c.M;
    double *A = (double *)malloc(rows * sizeof(double));
    double *B = (double *)malloc(rows * sizeof(double));
    if (!A || !B) { free(A); free(B); orc_free(&c); return ORC_ERR_NOMEM; }
    double ls = 0.0;
    st = orc_forward(&c, A, &ls);
    if (!st) {
        st = orc_end_row(&c, B);  /* B is overwritten by the backward pass below */
        const double le = st ? 0.0 : orc_end_logp(&c, A + (size_t)N * c.M, B);
        if (!st && !isfinite(le)) st = ORC_ERR_ZERO_PROB;
        else if (!st && loglik) *loglik = ls + le;
    }
    if (!st && (app || ext)) st = orc_backward(&c, B);
    if (!st && (app || ext)) st = orc_app(&c, A, B, app, ext, NULL);
    if (!st && ext) {
        for (int i = 0; i < N && !st; ++i) {
            double *e = ext + (size_t)i * q;
            double s = 0.0;
            for (int D = 0; D < q; ++D) s += e[D];
            if (!(s > 0.0)) st = ORC_ERR_ZERO_PROB;
            else
                for (int D = 0; D < q; ++D) e[D] /= s;
        }
    }
    free(A); free(B); orc_free(&c);
    return st;
}

/* Full decode with one codebook: APPs (N*q) and log P(Y). */
int orc_decode(int q, int n, const uint8_t *codebook, int N, double Pi, double Pd, double Ps,
               int I, int xmax, const uint8_t *rx, int64_t rho, const double *priors, int memo,
               double *app, double *loglik)
{
    return orc_decode_general(q, n, codebook, 0, N, Pi, Pd, Ps, I, xmax, rx, rho, priors, memo,
                              app, NULL, loglik, NULL, NULL);
}

/*
 * Normalised forward/backward metrics and forward normalisers, for tests of
 * the invariants.  A, B: (N+1)*M each; logc: N entries (log c_1..log c_N).
 */
int orc_forward_backward(int q, int n, const uint8_t *codebook, int N, double Pi, double Pd,
                         double Ps, int I, int xmax, const uint8_t *rx, int64_t rho,
                         const double *priors, double *A, double *B, double *logc)
{
    orc_ctx c;
    int st = orc_init(&c, q, n, codebook, 0, N, Pi, Pd, Ps, I, xmax, rx, rho, priors, 1, 0);
    if (st) { orc_free(&c); return st; }
    double ls = 0.0;
    st = orc_forward(&c, A, &ls);
    if (!st && logc) {
        /* recover each log c_i by re-running the normaliser sums */
        const int M = c.M;
        double *g = (double *)malloc((size_t)M * q * c.Mn * sizeof(double));
        double *an = (double *)malloc((size_t)M * sizeof(double));
        if (!g || !an) st = ORC_ERR_NOMEM;
        for (int i = 0; !st && i < N; ++i) {
            st = orc_gamma(&c, i, g, NULL);
            if (st) break;
            for (int m = 0; m < M; ++m) an[m] = 0.0;
            for (int mp = 0; mp < M; ++mp)
                for (int D = 0; D < q; ++D) {
                    const double *gd = g + ((size_t)mp * q + D) * c.Mn;
                    for (int k = 0; k < c.Mn; ++k) {
                        const int m = mp + k - n;
                        if (m >= 0 && m < M) an[m] += A[(size_t)i * M + mp] * gd[k];
                    }
                }
            double cs = 0.0;
            for (int m = 0; m < M; ++m) cs += an[m];
            logc[i] = log(cs);
        }
        free(g); free(an);
    }
    if (!st) st = orc_backward(&c, B);
    orc_free(&c);
    return st;
}

/*
 * log P(Y) and its gradient:
 *   dlogp_dchan[0..2] = d logP / d(Pi, Pd, Ps) with Pt = 1 - Pi - Pd and the
 *   drift limits held fixed (forward-mode dual numbers through the lattice
 *   and the forward pass);
 *   dlogp_dpriors[i*q + D] = d logP / d Pr{D_i = D} = Q_i(D) / Z_i.
 * Either output may be NULL.  codebooks / per_symbol as for orc_decode_general.
 */
int orc_loglik_grad_general(int q, int n, const uint8_t *codebooks, int per_symbol, int N,
                            double Pi, double Pd, double Ps, int I, int xmax, const uint8_t *rx,
                            int64_t rho, const double *priors, int memo, double *dlogp_dchan,
                            double *dlogp_dpriors, double *loglik, const double *phi0,
                            const double *phiN)
{
    orc_ctx c;
    int st = orc_init(&c, q, n, codebooks, per_symbol, N, Pi, Pd, Ps, I, xmax, rx, rho, priors,
                      memo, dlogp_dchan != NULL);
    if (st) { orc_free(&c); return st; }
    c.phi0 = phi0;
    c.phiN = phiN;
    const int M = c.M, Mn = c.Mn;
    double *bN = (double *)malloc((size_t)M * sizeof(double));
    double *a0 = (double *)malloc((size_t)M * sizeof(double));
    if (!bN || !a0) { free(bN); free(a0); orc_free(&c); return ORC_ERR_NOMEM; }
    double ls0 = 0.0;  /* log of the start row's sum (independent of the channel) */
    st = orc_start_row(&c, a0, &ls0);
    if (!st) st = orc_end_row(&c, bN);
    if (st) { free(bN); free(a0); orc_free(&c); return st; }
    if (dlogp_dchan) {
        dual *g = (dual *)malloc((size_t)M * q * Mn * sizeof(dual));
        dual *a = (dual *)malloc((size_t)M * sizeof(dual));
        dual *an = (dual *)malloc((size_t)M * sizeof(dual));
        if (!g || !a || !an) st = ORC_ERR_NOMEM;
        dual ls = d_const(ls0);
        if (!st)
            for (int m = 0; m < M; ++m) a[m] = d_const(a0[m]);
        for (int i = 0; !st && i < N; ++i) {
            st = orc_gamma_dual(&c, i, g);
            if (st) break;
            for (int m = 0; m < M; ++m) an[m] = d_const(0.0);
            for (int mp = 0; mp < M; ++mp)
                for (int D = 0; D < q; ++D) {
                    const dual *gd = g + ((size_t)mp * q + D) * Mn;
                    for (int k = 0; k < Mn; ++k) {
                        const int m = mp + k - n;
                        if (m >= 0 && m < M) an[m] = d_add(an[m], d_mul(a[mp], gd[k]));
                    }
                }
            dual cs = d_const(0.0);
            for (int m = 0; m < M; ++m) cs = d_add(cs, an[m]);
            if (!(cs.v > 0.0)) { st = ORC_ERR_ZERO_PROB; break; }
            for (int m = 0; m < M; ++m) a[m] = d_div(an[m], cs);
            ls = d_add(ls, d_log(cs));
        }
        if (!st) {
            dual e = d_const(0.0);  /* sum_m alpha_N(m) beta_N(m) */
            for (int m = 0; m < M; ++m) e = d_add(e, d_scale(a[m], bN[m]));
            if (!(e.v > 0.0)) st = ORC_ERR_ZERO_PROB;
            else {
                dual lp = d_add(ls, d_log(e));
                for (int k = 0; k < 3; ++k) dlogp_dchan[k] = lp.d[k];
                if (loglik) *loglik = lp.v - (double)((int64_t)n * N) * log(g_kappa);
            }
        }
        free(g); free(a); free(an);
        if (st) { free(bN); free(a0); orc_free(&c); return st; }
    }
    if (dlogp_dpriors || (!dlogp_dchan && loglik)) {
        const size_t rows = (size_t)(N + 1) * M;
        double *A = (double *)malloc(rows * sizeof(double));
        double *B = (double *)malloc(rows * sizeof(double));
        double *Z = (double *)malloc((size_t)N * sizeof(double));
        if (!A || !B || !Z) st = ORC_ERR_NOMEM;
        double ls = 0.0;
        if (!st) st = orc_forward(&c, A, &ls);
        if (!st && !dlogp_dchan && loglik) {
            const double le = orc_end_logp(&c, A + (size_t)N * M, bN);
            if (!isfinite(le)) st = ORC_ERR_ZERO_PROB;
            else *loglik = ls + le;
        }
        if (!st && dlogp_dpriors) st = orc_backward(&c, B);
        if (!st && dlogp_dpriors) st = orc_app(&c, A, B, NULL, dlogp_dpriors, Z);
        if (!st && dlogp_dpriors)
            for (int i = 0; i < N; ++i)
                for (int D = 0; D < q; ++D) dlogp_dpriors[(size_t)i * q + D] /= Z[i];
        free(A); free(B); free(Z);
    }
    free(bN); free(a0);
    orc_free(&c);
    return st;
}

/* log P(Y) and its gradient with one codebook for every symbol. */
int orc_loglik_grad(int q, int n, const uint8_t *codebook, int N, double Pi, double Pd,
                    double Ps, int I, int xmax, const uint8_t *rx, int64_t rho,
                    const double *priors, int memo, double *dlogp_dchan, double *dlogp_dpriors,
                    double *loglik)
{
    return orc_loglik_grad_general(q, n, codebook, 0, N, Pi, Pd, Ps, I, xmax, rx, rho, priors,
                                   memo, dlogp_dchan, dlogp_dpriors, loglik, NULL, NULL);
}
