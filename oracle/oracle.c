/*
 * oracle.c -- plain, slow FP64 CPU oracle for the CRN particle filter of
 * "Enhanced SMC^2: Leveraging Gradient Information from Differentiable
 * Particle Filters Within Langevin Proposals" (arXiv 2407.17296).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code;
 * it exists so that tests, the smoke check and the CPU-baseline leg of the
 * benchmark have an independent answer to compare the CUDA path against.  It
 * shares no source with the CUDA library.
 *
 * What it computes, step by step, in the paper's order:
 *   - common random numbers from Philox4x32-10 (Salmon et al., SC'11), keyed
 *     per (SMC^2 iteration, sample) as in Sec. I (one seed per sample and
 *     iteration) and drawn as Gaussians by Box-Muller;
 *   - the bootstrap particle filter: prior proposal (Eq. prior_proposal),
 *     weight update w_t = w_{t-1} g(y_t|x_t) (Eq. priorproposalweight),
 *     likelihood estimate (1/N_x) sum_j w_T^j (Eq. likelihood_pf_);
 *   - ESS-triggered resampling (Eq. ess) with the CRN resampler of App. B:
 *     normalised cumulative weights c^j, ancestor
 *     kappa_i = #{j : nu_i > c^j}, x' = x^{kappa}, w' = mean(w)
 *     (Eq. weightresample);
 *   - the forward-mode gradient of App. A/B: per particle the tangents
 *     dx/dtheta (Eqs. df, partialf, dxk) and dlog w/dtheta
 *     (Eqs. weightupdate, deriv_loglike), reset to the weighted mean at
 *     resampling (Eq. weightdiffresample and the display after it), and
 *     grad log p = sum_j w~_j dlog w_j (Eq. dloglik).
 *
 * Readings where the paper is garbled or silent:
 *   - log p-hat is the log of Eq. likelihood_pf_, i.e. LSE_j(log w_T^j) - log M
 *     with unnormalised initial weights w_0 = 1 (Eq. likelihood_pf as printed,
 *     a mean of log-weights, is not an estimate of the log-likelihood);
 *   - ancestor index: a_i = min{j : c_j >= tau_i} (0-based, c_{M-1} := 1), the
 *     0-based form of the strict "nu > c^j" count of App. B;
 *   - systematic resampling uses tau_i = (i + nu)/M with one nu per step;
 *     multinomial (the paper's scheme) uses one nu_i per particle;
 *   - resample before step t when ESS_{t-1} < ess_frac * M (Eq. ess criterion
 *     with the fraction configurable); never before step 1.
 *
 * Random-number layout (shared definition with the CUDA path, not shared code):
 *   key  = (seed_lo ^ iter, seed_hi ^ row)
 *   ctr  = (t, call, stream, 0)
 *   stream 0: propagation noise at step t (normal index n = j*dx + k, call = n/4)
 *   stream 1: resampling uniforms before step t (systematic: call 0 word 0;
 *             multinomial: particle i uses call i/4, word i%4)
 *   stream 2: initial state noise (t = 0, normal index n = j*dx + k)
 *   stream 3: outer-sampler Gaussians (t = 0, normal index d)
 *   stream 4: outer-sampler resampling uniform (t = 0, call 0, word 0), with
 *             key (seed_lo ^ iter, seed_hi)
 *   uniform on (0,1]: ((u >> 8) + 1) * 2^-24;  on [0,1): (u >> 8) * 2^-24.
 *   Box-Muller on words (u0,u1): r = sqrt(-2 ln U(0,1](u0)), phi = 2 pi U[0,1)(u1),
 *   z0 = r cos phi, z1 = r sin phi; words (u2,u3) likewise give z2, z3.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_TWO_PI 6.283185307179586476925286766559
#define OR_LOG_2PI 1.8378770664093454835606594728112

enum { OR_LG_DIAG = 0, OR_SV = 1, OR_LG_OPT = 2 };
enum { OR_SYSTEMATIC = 0, OR_MULTINOMIAL = 1 };
enum { OR_STREAM_PROP = 0, OR_STREAM_RESAMPLE = 1, OR_STREAM_INIT = 2,
       OR_STREAM_OUTER_XI = 3, OR_STREAM_OUTER_NU = 4 };

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from the published description of the algorithm.          */
/* ------------------------------------------------------------------------ */

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u; /* golden ratio Weyl increment */
            k1 += 0xBB67AE85u; /* sqrt(3)-1 Weyl increment */
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static double u_open01(uint32_t u) { return ((double)(u >> 8) + 1.0) * (1.0 / 16777216.0); }
static double u_half01(uint32_t u) { return (double)(u >> 8) * (1.0 / 16777216.0); }

/* Four standard normals from one Philox call by Box-Muller. */
static void box_muller4(const uint32_t w[4], double z[4])
{
    double r01 = sqrt(-2.0 * log(u_open01(w[0])));
    double p01 = OR_TWO_PI * u_half01(w[1]);
    double r23 = sqrt(-2.0 * log(u_open01(w[2])));
    double p23 = OR_TWO_PI * u_half01(w[3]);
    z[0] = r01 * cos(p01);
    z[1] = r01 * sin(p01);
    z[2] = r23 * cos(p23);
    z[3] = r23 * sin(p23);
}

static void make_key(uint64_t seed, uint32_t iter, uint32_t row, uint32_t key[2])
{
    key[0] = (uint32_t)(seed & 0xFFFFFFFFu) ^ iter;
    key[1] = (uint32_t)(seed >> 32) ^ row;
}

/* n standard normals with indices 0..n-1 for (key, t, stream). */
static void normals(const uint32_t key[2], uint32_t t, uint32_t stream, long n, double* out)
{
    long calls = (n + 3) / 4;
    for (long c = 0; c < calls; ++c) {
        uint32_t ctr[4] = {t, (uint32_t)c, stream, 0u}, w[4];
        double z[4];
        oracle_philox4x32_10(ctr, key, w);
        box_muller4(w, z);
        for (int q = 0; q < 4; ++q)
            if (4 * c + q < n) out[4 * c + q] = z[q];
    }
}

/* Exported helpers so the Python side of the oracle uses the same generator. */
void oracle_normals(uint64_t seed, uint32_t iter, uint32_t row, uint32_t t, uint32_t stream,
                    long n, double* out)
{
    uint32_t key[2];
    make_key(seed, iter, row, key);
    normals(key, t, stream, n, out);
}

double oracle_uniform_open(uint64_t seed, uint32_t iter, uint32_t row, uint32_t t,
                           uint32_t stream, uint32_t call, int word)
{
    uint32_t key[2], ctr[4] = {t, call, stream, 0u}, w[4];
    make_key(seed, iter, row, key);
    oracle_philox4x32_10(ctr, key, w);
    return u_open01(w[word & 3]);
}

/* ------------------------------------------------------------------------ */
/* State-space model families (Sec. II, Eqs. xt and yt).                    */
/*                                                                          */
/* LG_DIAG: theta = (a[dx], log q[dx], log r[dy]),                          */
/*   x_0 ~ N(0, I), x_t = diag(a) x_{t-1} + diag(exp(log q)) eps_t,          */
/*   y_t ~ N(H x_t, diag(exp(log r))^2).                                    */
/* SV:      theta = (mu, atanh phi, log sigma),                             */
/*   x_0 = mu + sigma/sqrt(1-phi^2) eps_0,                                  */
/*   x_t = mu + phi (x_{t-1} - mu) + sigma eta_t, y_t ~ N(0, exp(x_t)).     */
/* LG_OPT:  the linear-Gaussian model of Sec. IV-A, theta = (mu, phi, sigma) */
/*   in their own units, x_0 ~ N(0, 1), x_t | x_{t-1} ~ N(mu x_{t-1}, phi^2), */
/*   y_t | x_t ~ N(x_t, sigma^2), filtered with the "optimal" proposal       */
/*   q(x_t | x_{t-1}, y_t) = N(rho^2 (y_t/sigma^2 + mu x_{t-1}/phi^2), rho^2),*/
/*   1/rho^2 = 1/phi^2 + 1/sigma^2, whose weight (Eq. weightupdate) is       */
/*   p(y_t | x_{t-1}) = N(y_t; mu x_{t-1}, phi^2 + sigma^2).                 */
/* ------------------------------------------------------------------------ */

typedef struct {
    int family, dx, dy, D;
    const double* H; /* dy x dx row-major; NULL means identity (dx == dy) */
} or_model;

static double H_at(const or_model* m, int r, int c)
{
    if (m->H) return m->H[r * m->dx + c];
    return r == c ? 1.0 : 0.0;
}

/*
 * Initial particle x_0 from its noise eps[dx], and dx_0/dtheta (dx x D, row-major).
 */
static void model_init(const or_model* m, const double* th, const double* eps, double* x, double* J)
{
    int dx = m->dx, D = m->D;
    memset(J, 0, sizeof(double) * dx * D);
    if (m->family == OR_LG_DIAG || m->family == OR_LG_OPT) {
        for (int k = 0; k < dx; ++k) x[k] = eps[k];
    } else {
        double mu = th[0], phi = tanh(th[1]), sig = exp(th[2]);
        double sd0 = sig / sqrt(1.0 - phi * phi);
        x[0] = mu + sd0 * eps[0];
        J[0] = 1.0;                    /* d/dmu */
        J[1] = phi * sd0 * eps[0];     /* d/d atanh(phi): sd0 = sigma cosh(psi), d cosh = sinh = phi cosh */
        J[2] = sd0 * eps[0];           /* d/d log sigma */
    }
}

/*
 * Reparameterised transition x_new = f(x, theta, eps) (Eq. reparam_epsilon)
 * with its partial derivatives Fx = df/dx (dx x dx) and Ft = df/dtheta (dx x D).
 */
static void model_transition(const or_model* m, const double* th, const double* x, const double* eps,
                             double* xn, double* Fx, double* Ft)
{
    int dx = m->dx, D = m->D;
    memset(Fx, 0, sizeof(double) * dx * dx);
    memset(Ft, 0, sizeof(double) * dx * D);
    if (m->family == OR_LG_DIAG) {
        for (int k = 0; k < dx; ++k) {
            double a = th[k], q = exp(th[dx + k]);
            xn[k] = a * x[k] + q * eps[k];
            Fx[k * dx + k] = a;
            Ft[k * D + k] = x[k];            /* d/da_k */
            Ft[k * D + dx + k] = q * eps[k]; /* d/dlog q_k */
        }
    } else {
        double mu = th[0], phi = tanh(th[1]), sig = exp(th[2]);
        xn[0] = mu + phi * (x[0] - mu) + sig * eps[0];
        Fx[0] = phi;
        Ft[0] = 1.0 - phi;                        /* d/dmu */
        Ft[1] = (1.0 - phi * phi) * (x[0] - mu);  /* d/d atanh(phi) */
        Ft[2] = sig * eps[0];                     /* d/d log sigma */
    }
}

/*
 * log g(y|x, theta) (Eq. L) with its partials Lx = dL/dx (dx) and Lt = dL/dtheta (D),
 * the ingredients of Eq. deriv_loglike.
 */
static double model_loglik(const or_model* m, const double* th, const double* x, const double* y,
                           double* Lx, double* Lt)
{
    int dx = m->dx, dy = m->dy, D = m->D;
    memset(Lx, 0, sizeof(double) * dx);
    memset(Lt, 0, sizeof(double) * D);
    double L = 0.0;
    if (m->family == OR_LG_DIAG) {
        for (int r = 0; r < dy; ++r) {
            double lr = th[2 * dx + r];
            double prec = exp(-2.0 * lr);
            double h = 0.0;
            for (int c = 0; c < dx; ++c) h += H_at(m, r, c) * x[c];
            double e = y[r] - h;
            L += -0.5 * (e * e * prec + 2.0 * lr + OR_LOG_2PI);
            for (int c = 0; c < dx; ++c) Lx[c] += e * prec * H_at(m, r, c);
            Lt[2 * dx + r] = e * e * prec - 1.0;
        }
    } else {
        double v = exp(-x[0]);
        L = -0.5 * (OR_LOG_2PI + x[0] + y[0] * y[0] * v);
        Lx[0] = -0.5 + 0.5 * y[0] * y[0] * v;
    }
    return L;
}

/*
 * LG_OPT weight log p(y | x_prev) = log N(y; mu x_prev, phi^2 + sigma^2) with its partials
 * Lx = d/dx_prev and Lt = d/dtheta.
 */
static double opt_weight(const double* th, double xp, double y, double* Lx, double* Lt)
{
    double mu = th[0], phi = th[1], sig = th[2];
    double s2 = phi * phi + sig * sig;
    double r = y - mu * xp;
    double L = -0.5 * (OR_LOG_2PI + log(s2) + r * r / s2);
    double dL_ds2 = -0.5 / s2 + 0.5 * r * r / (s2 * s2);
    *Lx = mu * r / s2;
    Lt[0] = xp * r / s2;
    Lt[1] = dL_ds2 * 2.0 * phi;
    Lt[2] = dL_ds2 * 2.0 * sig;
    return L;
}

/*
 * LG_OPT proposal x = (phi^2 y + sigma^2 mu x_prev)/s2 + rho eps, s2 = phi^2 + sigma^2,
 * rho = phi sigma / sqrt(s2), with Fx = dx/dx_prev and Ft = dx/dtheta.
 */
static void opt_transition(const double* th, double xp, double y, double eps, double* xn, double* Fx,
                           double* Ft)
{
    double mu = th[0], phi = th[1], sig = th[2];
    double p2 = phi * phi, q2 = sig * sig, s2 = p2 + q2;
    double rho = phi * sig / sqrt(s2);
    double mean = (p2 * y + q2 * mu * xp) / s2;
    *xn = mean + rho * eps;
    *Fx = q2 * mu / s2;
    /* d mean/d phi = (2 phi y s2 - (p2 y + q2 mu xp) 2 phi)/s2^2 = 2 phi q2 (y - mu xp)/s2^2 */
    /* d mean/d sig = (2 sig mu xp s2 - (p2 y + q2 mu xp) 2 sig)/s2^2 = 2 sig p2 (mu xp - y)/s2^2 */
    /* d rho/d phi = sig^3/s2^(3/2), d rho/d sig = phi^3/s2^(3/2) */
    double s32 = s2 * sqrt(s2);
    Ft[0] = q2 * xp / s2;
    Ft[1] = 2.0 * phi * q2 * (y - mu * xp) / (s2 * s2) + sig * q2 / s32 * eps;
    Ft[2] = 2.0 * sig * p2 * (mu * xp - y) / (s2 * s2) + phi * p2 / s32 * eps;
}

/* ------------------------------------------------------------------------ */
/* The CRN particle filter with forward-mode gradient.                      */
/* ------------------------------------------------------------------------ */

/* stats[] slots */
enum {
    ST_NEAR_TIES = 0,      /* ancestor decisions whose cumulative weight lies within band of the threshold */
    ST_TIE_FOLLOWED,       /* of those, hint differed from own decision and was followed */
    ST_NONTIE_MISMATCH,    /* hint differed from own decision outside the band (a parity failure) */
    ST_FLAG_TIES,          /* resample decisions within band that differed from the hint */
    ST_FLAG_MISMATCH,      /* resample decisions that differed from the hint outside the band */
    ST_RESAMPLE_STEPS,     /* number of steps that resampled */
    ST_BAD_HINT,           /* hint ancestor out of range */
    ST_TIE_COND,           /* followed differences outside band but inside the conditioned band */
    ST_COUNT
};

static double logsumexp(const double* v, int n)
{
    double mx = -INFINITY;
    for (int i = 0; i < n; ++i) if (v[i] > mx) mx = v[i];
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += exp(v[i] - mx);
    return mx + log(s);
}

/* smallest j with c[j] >= tau (c non-decreasing, c[M-1] == 1) */
static int first_at_least(const double* c, int M, double tau)
{
    for (int j = 0; j < M; ++j)
        if (c[j] >= tau) return j;
    return M - 1;
}

/*
 * oracle_pf: one CRN-PF run for one theta.
 *
 *   m, theta[D], y[T*dy] (FP32 observations, shared by both implementations)
 *   T, M, seed/iter/row -> Philox key
 *   scheme: 0 systematic, 1 multinomial; ess_frac: resample when ESS < ess_frac*M
 *   want_grad: carry the forward-mode tangents
 *   hint_anc[T*M], hint_flag[T] (may be NULL): decisions taken elsewhere.
 *     replay = 1: use them everywhere (log p-hat becomes a smooth function of theta).
 *     replay = 0 ("follow"): use the oracle's own decision unless it differs from
 *     the hint; differences are classified against the band (|c - tau| < band for
 *     ancestors, |ESS/(ess_frac*M) - 1| < band for the resample flag) and counted,
 *     and the hint is then followed so that later steps stay comparable.
 *     band_rel >= 0 widens both bands to max(band, band_rel * L) where L is the sum, over
 *     the steps since the last resampling, of the largest |log g| of the step: an FP32
 *     evaluation of log w then carries an absolute error of order 2^-24 L, which moves
 *     the cumulative weights by about as much.  Differences inside the widened band but
 *     outside the base band are counted separately (ST_TIE_COND).
 *   outputs: loglik, grad[D] (if want_grad), anc_out[T*M], flag_out[T] (may be NULL),
 *     stats[ST_COUNT], worst[1] = largest |c - tau| distance of a non-tie mismatch.
 * Row t-1 of the tapes describes resampling before step t (row 0 is never used).
 * Returns 0, or -1 on bad arguments / allocation failure.
 */
int oracle_pf(int family, int dx, int dy, int D, const double* H,
              const double* theta, const float* y, int T, int M,
              uint64_t seed, uint32_t iter, uint32_t row,
              int scheme, double ess_frac, int want_grad,
              const uint16_t* hint_anc, const uint8_t* hint_flag, int replay, double band, double flag_band,
              double band_rel, double* loglik, double* grad, uint16_t* anc_out, uint8_t* flag_out,
              long long* stats, double* worst)
{
    or_model m = {family, dx, dy, D, H};
    if (T < 1 || M < 1 || dx < 1 || dy < 1 || D < 1) return -1;
    if (family == OR_SV && (dx != 1 || dy != 1 || D != 3)) return -1;
    if (family == OR_LG_DIAG && D != 2 * dx + dy) return -1;
    if (family == OR_LG_OPT && (dx != 1 || dy != 1 || D != 3)) return -1;
    if (family < OR_LG_DIAG || family > OR_LG_OPT) return -1;
    if (replay && (!hint_anc || !hint_flag)) return -1;

    long long st[ST_COUNT];
    memset(st, 0, sizeof(st));
    double worst_dist = 0.0;

    uint32_t key[2];
    make_key(seed, iter, row, key);

    size_t nJ = (size_t)dx * D;
    double* x = calloc((size_t)M * dx, sizeof(double));
    double* xn = calloc((size_t)M * dx, sizeof(double));
    double* J = calloc((size_t)M * nJ, sizeof(double));
    double* Jn = calloc((size_t)M * nJ, sizeof(double));
    double* lw = calloc((size_t)M, sizeof(double));
    double* g = calloc((size_t)M * D, sizeof(double));
    double* gn = calloc((size_t)M * D, sizeof(double));
    double* eps = calloc((size_t)M * dx + 4, sizeof(double));
    double* c = calloc((size_t)M, sizeof(double));
    double* wt = calloc((size_t)M, sizeof(double));
    double* nu = calloc((size_t)M, sizeof(double));
    int* anc = calloc((size_t)M, sizeof(int));
    double* Fx = calloc((size_t)dx * dx, sizeof(double));
    double* Ft = calloc((size_t)dx * D, sizeof(double));
    double* Lx = calloc((size_t)dx, sizeof(double));
    double* Lt = calloc((size_t)D, sizeof(double));
    double* yt = calloc((size_t)dy, sizeof(double));
    int ok = x && xn && J && Jn && lw && g && gn && eps && c && wt && nu && anc && Fx && Ft && Lx && Lt && yt;
    if (!ok) {
        free(x); free(xn); free(J); free(Jn); free(lw); free(g); free(gn); free(eps); free(c);
        free(wt); free(nu); free(anc); free(Fx); free(Ft); free(Lx); free(Lt); free(yt);
        return -1;
    }
    if (anc_out) memset(anc_out, 0, sizeof(uint16_t) * (size_t)T * M);
    if (flag_out) memset(flag_out, 0, (size_t)T);

    /* t = 0: x_0 from the initial distribution, unnormalised weights w_0 = 1. */
    normals(key, 0u, OR_STREAM_INIT, (long)M * dx, eps);
    for (int j = 0; j < M; ++j) {
        model_init(&m, theta, eps + (size_t)j * dx, x + (size_t)j * dx, J + (size_t)j * nJ);
        lw[j] = 0.0;
    }

    int resample_next = 0;
    double ess_prev = (double)M;
    double lacc = 0.0; /* sum of max |log g| per step since the last resampling */
    for (int t = 1; t <= T; ++t) {
        /* ---- resampling decision and CRN resampling before step t (App. B) ---- */
        if (t >= 2) {
            int own = resample_next;
            int use = own;
            const double wide = band_rel * lacc;
            if (hint_flag) {
                int h = hint_flag[t - 1] ? 1 : 0;
                if (replay) {
                    use = h;
                } else if (h != own) {
                    double rel = fabs(ess_prev / (ess_frac * M) - 1.0);
                    if (rel < flag_band) st[ST_FLAG_TIES]++;
                    else if (rel < wide) st[ST_TIE_COND]++;
                    else st[ST_FLAG_MISMATCH]++;
                    use = h;
                }
            }
            if (use) {
                st[ST_RESAMPLE_STEPS]++;
                if (flag_out) flag_out[t - 1] = 1;
                /* normalised weights and their cumulative sums c_j */
                double L = logsumexp(lw, M);
                double run = 0.0;
                for (int j = 0; j < M; ++j) wt[j] = exp(lw[j] - L);
                for (int j = 0; j < M; ++j) { run += wt[j]; c[j] = run; }
                for (int j = 0; j < M; ++j) c[j] = c[j] / run;
                c[M - 1] = 1.0;
                /* thresholds */
                if (scheme == OR_SYSTEMATIC) {
                    double v = 0.0;
                    {
                        uint32_t ctr[4] = {(uint32_t)t, 0u, OR_STREAM_RESAMPLE, 0u}, w[4];
                        oracle_philox4x32_10(ctr, key, w);
                        v = u_open01(w[0]);
                    }
                    for (int i = 0; i < M; ++i) nu[i] = ((double)i + v) / (double)M;
                } else {
                    for (int i = 0; i < M; ++i) {
                        uint32_t ctr[4] = {(uint32_t)t, (uint32_t)(i / 4), OR_STREAM_RESAMPLE, 0u}, w[4];
                        oracle_philox4x32_10(ctr, key, w);
                        nu[i] = u_open01(w[i % 4]);
                    }
                }
                for (int i = 0; i < M; ++i) {
                    int own_a = first_at_least(c, M, nu[i]);
                    /* near-tie: another index is admissible within the band */
                    int near = (c[own_a] - nu[i] < band) || (own_a > 0 && nu[i] - c[own_a - 1] <= band);
                    if (near) st[ST_NEAR_TIES]++;
                    int a = own_a;
                    if (hint_anc) {
                        int h = (int)hint_anc[(size_t)(t - 1) * M + i];
                        if (h < 0 || h >= M) {
                            st[ST_BAD_HINT]++;
                        } else if (replay) {
                            a = h;
                        } else if (h != own_a) {
                            /* distance by which h violates "c_{h-1} < tau <= c_h" */
                            double lo = (h > 0) ? c[h - 1] : 0.0;
                            double d1 = nu[i] - c[h];     /* > 0 if c_h < tau */
                            double d2 = lo - nu[i];       /* >= 0 if c_{h-1} >= tau */
                            double dist = d1 > d2 ? d1 : d2;
                            if (dist < band) st[ST_TIE_FOLLOWED]++;
                            else if (dist < wide) st[ST_TIE_COND]++;
                            else {
                                st[ST_NONTIE_MISMATCH]++;
                                if (dist > worst_dist) worst_dist = dist;
                            }
                            a = h;
                        }
                    }
                    anc[i] = a;
                    if (anc_out) anc_out[(size_t)(t - 1) * M + i] = (uint16_t)a;
                }
                /* x' = x^{kappa}, dx'/dtheta = dx^{kappa}/dtheta */
                for (int i = 0; i < M; ++i) {
                    memcpy(xn + (size_t)i * dx, x + (size_t)anc[i] * dx, sizeof(double) * dx);
                    memcpy(Jn + (size_t)i * nJ, J + (size_t)anc[i] * nJ, sizeof(double) * nJ);
                }
                { double* s = x; x = xn; xn = s; s = J; J = Jn; Jn = s; }
                /* w' = (1/M) sum_j w_j for every particle; dlog w' = sum_j w~_j dlog w_j */
                double lw_new = L - log((double)M);
                if (want_grad) {
                    for (int d = 0; d < D; ++d) {
                        double s = 0.0;
                        for (int j = 0; j < M; ++j) s += wt[j] * g[(size_t)j * D + d];
                        for (int i = 0; i < M; ++i) gn[(size_t)i * D + d] = s;
                    }
                    double* s = g; g = gn; gn = s;
                }
                for (int i = 0; i < M; ++i) lw[i] = lw_new;
                lacc = 0.0;
            }
        }

        /* ---- propagate with the prior proposal and reweight (Eq. priorproposalweight) ---- */
        normals(key, (uint32_t)t, OR_STREAM_PROP, (long)M * dx, eps);
        for (int r = 0; r < dy; ++r) yt[r] = (double)y[(size_t)(t - 1) * dy + r];
        double step_max_abs = 0.0;
        for (int j = 0; j < M; ++j) {
            double* xj = x + (size_t)j * dx;
            double* xnj = xn + (size_t)j * dx;
            if (family == OR_LG_OPT) {
                /* optimal proposal: the weight depends on the previous state only */
                double Lj = opt_weight(theta, xj[0], yt[0], Lx, Lt);
                opt_transition(theta, xj[0], yt[0], eps[j], xnj, Fx, Ft);
                lw[j] += Lj;
                if (fabs(Lj) > step_max_abs) step_max_abs = fabs(Lj);
                if (want_grad) {
                    double* Jj = J + (size_t)j * nJ;
                    double* Jnj = Jn + (size_t)j * nJ;
                    for (int d = 0; d < D; ++d) {
                        g[(size_t)j * D + d] += Lt[d] + Lx[0] * Jj[d];   /* through x_{t-1} */
                        Jnj[d] = Ft[d] + Fx[0] * Jj[d];
                    }
                }
                continue;
            }
            model_transition(&m, theta, xj, eps + (size_t)j * dx, xnj, Fx, Ft);
            double Lj = model_loglik(&m, theta, xnj, yt, Lx, Lt);
            lw[j] += Lj;
            if (fabs(Lj) > step_max_abs) step_max_abs = fabs(Lj);
            if (want_grad) {
                double* Jj = J + (size_t)j * nJ;
                double* Jnj = Jn + (size_t)j * nJ;
                /* dx_t/dtheta = df/dx dx_{t-1}/dtheta + df/dtheta  (Eq. dxk) */
                for (int k = 0; k < dx; ++k)
                    for (int d = 0; d < D; ++d) {
                        double s = Ft[k * D + d];
                        for (int l = 0; l < dx; ++l) s += Fx[k * dx + l] * Jj[l * D + d];
                        Jnj[k * D + d] = s;
                    }
                /* dlog w_t = dlog w_{t-1} + dL/dx dx_t/dtheta + dL/dtheta  (Eqs. weightupdate, deriv_loglike) */
                for (int d = 0; d < D; ++d) {
                    double s = Lt[d];
                    for (int k = 0; k < dx; ++k) s += Lx[k] * Jnj[k * D + d];
                    g[(size_t)j * D + d] += s;
                }
            }
        }
        { double* s = x; x = xn; xn = s; }
        if (want_grad) { double* s = J; J = Jn; Jn = s; }
        lacc += step_max_abs;

        /* ---- ESS of the new weights (Eq. ess) for the next decision ---- */
        if (t < T) {
            double L = logsumexp(lw, M);
            double s2 = 0.0;
            for (int j = 0; j < M; ++j) { double w = exp(lw[j] - L); s2 += w * w; }
            ess_prev = 1.0 / s2;
            resample_next = ess_prev < ess_frac * (double)M;
        }
    }

    /* log p-hat = log((1/M) sum_j w_T^j)  (Eq. likelihood_pf_) */
    double L = logsumexp(lw, M);
    *loglik = L - log((double)M);
    if (want_grad && grad) {
        /* grad = sum_j w~_j dlog w_j  (Eq. dloglik) */
        for (int d = 0; d < D; ++d) {
            double s = 0.0;
            for (int j = 0; j < M; ++j) s += exp(lw[j] - L) * g[(size_t)j * D + d];
            grad[d] = s;
        }
    }
    if (stats) memcpy(stats, st, sizeof(st));
    if (worst) *worst = worst_dist;

    free(x); free(xn); free(J); free(Jn); free(lw); free(g); free(gn); free(eps); free(c);
    free(wt); free(nu); free(anc); free(Fx); free(Ft); free(Lx); free(Lt); free(yt);
    return 0;
}

/*
 * Ancestors for given normalised weights and uniforms, straight from the
 * definition a_i = min{j : c_j >= tau_i} (exported for the resampling pins).
 */
void oracle_ancestors(const double* w, int M, const double* tau, int n_tau, int* out)
{
    double* c = malloc(sizeof(double) * (size_t)M);
    if (!c) return;
    double run = 0.0, tot = 0.0;
    for (int j = 0; j < M; ++j) tot += w[j];
    for (int j = 0; j < M; ++j) { run += w[j]; c[j] = run / tot; }
    c[M - 1] = 1.0;
    for (int i = 0; i < n_tau; ++i) out[i] = first_at_least(c, M, tau[i]);
    free(c);
}
