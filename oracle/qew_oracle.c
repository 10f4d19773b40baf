/*
 * qew_oracle.c -- plain, slow FP64 CPU oracle for the explicit-Euler relaxation of the
 * discretised 1D quenched Edwards-Wilkinson (qEW) equation of Ferrero, Bustingorry and
 * Kolton, "Non-steady relaxation and critical exponents at the depinning transition"
 * (arXiv:1211.7275).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call this
 * file: only the tests, the smoke check and the CPU-baseline leg of the benchmark use it.
 * It shares no code, header, table or constant generator with the CUDA path.
 *
 * What it computes (one periodic chain s of L sites, FP64 state u_i):
 *   Eq. 1 with eta = c = 1, discretised in x with dx = 1 and periodic boundary conditions
 *   (Sec. III.B): du_i/dt = u_{i+1} + u_{i-1} - 2 u_i + f + F_p(i, u_i), integrated with
 *   the explicit Euler method, all forces taken from the old state (synchronous update).
 *   The pinning force is built from uncorrelated random numbers drawn at the integer
 *   points (i, n) of the (x, u) plane and interpolated in u (Sec. III.B; Sec. IV.C list of
 *   disorder cases):
 *     RF (random field, Case 4):  F = (1 - d) R(i, n) + d R(i, n + 1),  R ~ N(0, 1)
 *     RB (random bond, cubic):    F = -dV/du, V the uniform Catmull-Rom spline through
 *                                 V(i, n-1 .. n+2),  V ~ U(-1, 1)          (Case 2)
 *     NONE:                       F = 0 (disorder-free line; closed-form tests)
 *     RB-G linear (Case 3):       F = -dV/du of the linear spline through the Gaussian
 *                                 potential values G(i, n), G(i, n+1):  F = G(n) - G(n+1),
 *                                 constant inside a cell and discontinuous at the integers
 *     RB-G cubic (Case 1):        F = -dV/du, V the Catmull-Rom spline through
 *                                 G(i, n-1 .. n+2),  G ~ N(0, 1)
 *   with n = floor(u), d = u - n.
 *   Periodic disorder (the L x M system of Sec. III.B): with a period M > 0 every node index n
 *   is taken mod M (in [0, M)) before it keys the generator, so the disorder repeats in u
 *   with period M; M = 0 leaves it aperiodic (the memory-free runs of Sec. IV.D).
 *   Observables (Sec. II, Eqs. 3-5): v = f + (1/L) sum_i F_i at the observed state (the
 *   periodic Laplacian sums to zero), ubar = (1/L) sum_i u_i, w2 = (1/L) sum_i (u_i-ubar)^2.
 *   Flat start u_i(0) = 0 (Sec. II).
 *
 * Random numbers (the paper does not say which generator it used; readings chosen here):
 *   Philox4x32-10 of Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as
 *   1, 2, 3" (SC'11), written from that paper's definition: key (lo32(seed), hi32(seed)),
 *   counter (i, (uint32) n, s, tag) with tag 0 for RF forces, 1 for uniform RB potentials
 *   and 2 for Gaussian RB potentials (shared by Cases 1 and 3: the same potential values,
 *   interpolated two ways).
 *   Uniforms U_k = (x_k + 1/2) 2^-32 from output words x_0, x_1.
 *   R, G = sqrt(-2 ln U_1) cos(2 pi U_2)   (Box and Muller 1958, cosine branch)
 *   V = (x_0 + 1/2) 2^-31 - 1.
 *
 * FP32 node model (oracle_run with node_f32 = 1): the same dynamics, in FP64, with every
 * disorder value rounded to the nearest FP32 number before it enters the force.  This is the
 * exact dynamics of the disorder as any FP32 store of it holds it; comparing it with the exact
 * run measures how far the rounding of the disorder alone moves the line (near the depinning
 * threshold it is amplified), which is the floor of every FP32 implementation.
 *
 * Build: gcc -O2 -std=c11 -fPIC -shared -ffp-contract=off (no fused multiply-add, so the
 * rounding sequence is the one written here on every host).
 */
#define _GNU_SOURCE
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define QO_RF 0
#define QO_RB 1
#define QO_NONE 2
#define QO_RBG_LINEAR 3
#define QO_RBG_CUBIC 4

/* ------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11).                                                */
/* One round: two 32x32->64 multiplications of words 0 and 2 by the round multipliers;   */
/* the new words are (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0)).   */
/* The key is bumped by the Weyl constants between rounds.                              */
/* ------------------------------------------------------------------------------------ */
static const uint32_t PHILOX_M0 = 0xD2511F53u;
static const uint32_t PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u;
static const uint32_t PHILOX_W1 = 0xBB67AE85u;

static void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

void oracle_philox4x32_10(const uint32_t* ctr, const uint32_t* key, int64_t n_blocks, uint32_t* out)
{
    for (int64_t b = 0; b < n_blocks; ++b)
        philox4x32_10(ctr + 4 * b, key + 2 * b, out + 4 * b);
}

/* The four output words for the disorder value at integer point (i, n) of chain s. */
static void disorder_words(uint64_t seed, uint32_t s, int64_t i, int64_t n, uint32_t tag, uint32_t w[4])
{
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)(int32_t)n, s, tag};
    philox4x32_10(ctr, key, w);
}

/* Node index of a disorder periodic in u with period M (the L x M system of Sec. III.B):
   n mod M in [0, M); M <= 0 leaves the disorder aperiodic. */
static int64_t wrap_node(int64_t n, int64_t period)
{
    if (period <= 0)
        return n;
    int64_t r = n % period;
    return r < 0 ? r + period : r;
}

/* N(0, 1) value from two output words: Box-Muller, cosine branch. */
static double box_muller(const uint32_t w[4])
{
    double u1 = ((double)w[0] + 0.5) * 0x1p-32;
    double u2 = ((double)w[1] + 0.5) * 0x1p-32;
    double r = sqrt(-2.0 * log(u1));
    return r * cos(2.0 * M_PI * u2);
}

/* RF force value R(s, i, n) ~ N(0, 1). */
static double rf_value(uint64_t seed, uint32_t s, int64_t i, int64_t n)
{
    uint32_t w[4];
    disorder_words(seed, s, i, n, 0u, w);
    return box_muller(w);
}

/* Gaussian RB potential value G(s, i, n) ~ N(0, 1) (Cases 1 and 3). */
static double rbg_value(uint64_t seed, uint32_t s, int64_t i, int64_t n)
{
    uint32_t w[4];
    disorder_words(seed, s, i, n, 2u, w);
    return box_muller(w);
}

/* RB potential value V(s, i, n) ~ U(-1, 1). */
static double rb_value(uint64_t seed, uint32_t s, int64_t i, int64_t n)
{
    uint32_t w[4];
    disorder_words(seed, s, i, n, 1u, w);
    return ((double)w[0] + 0.5) * 0x1p-31 - 1.0;
}

/* Potential value at an integer point for the RB kinds. */
static double potential_value(int kind, uint64_t seed, uint32_t s, int64_t i, int64_t n, int64_t period)
{
    n = wrap_node(n, period);
    return kind == QO_RB ? rb_value(seed, s, i, n) : rbg_value(seed, s, i, n);
}

/* A disorder value as the force sees it: exact, or rounded to the nearest FP32 number (the
   FP32 node model; the conversion rounds to nearest, ties to even). */
static double node_value(double v, int node_f32)
{
    return node_f32 ? (double)(float)v : v;
}

/* Pinning force at site i of chain s and displacement u (Sec. III.B, Sec. IV.C); with
   node_f32 every disorder value is rounded to FP32 first. */
static double pinning_force_nodes(int kind, uint64_t seed, uint32_t s, int64_t i, double u, int64_t period,
                                  int node_f32)
{
    if (kind == QO_NONE)
        return 0.0;
    double fl = floor(u);
    int64_t n = (int64_t)fl;
    double d = u - fl;
    if (kind == QO_RF) {
        double r0 = node_value(rf_value(seed, s, i, wrap_node(n, period)), node_f32);
        double r1 = node_value(rf_value(seed, s, i, wrap_node(n + 1, period)), node_f32);
        return (1.0 - d) * r0 + d * r1;
    }
    if (kind == QO_RBG_LINEAR) {
        /* V(u) = (1 - d) G(n) + d G(n+1) on [n, n+1), so -dV/du = G(n) - G(n+1) */
        return node_value(rbg_value(seed, s, i, wrap_node(n, period)), node_f32) -
               node_value(rbg_value(seed, s, i, wrap_node(n + 1, period)), node_f32);
    }
    /* RB / RB-G cubic: V(u) on [n, n+1] is the uniform Catmull-Rom cubic through
       p0..p3 = V(n-1..n+2):
       V(d) = 1/2 [2 p1 + (p2 - p0) d + (2p0 - 5p1 + 4p2 - p3) d^2 + (-p0 + 3p1 - 3p2 + p3) d^3]
       and F = -dV/du. */
    double p0 = node_value(potential_value(kind, seed, s, i, n - 1, period), node_f32);
    double p1 = node_value(potential_value(kind, seed, s, i, n, period), node_f32);
    double p2 = node_value(potential_value(kind, seed, s, i, n + 1, period), node_f32);
    double p3 = node_value(potential_value(kind, seed, s, i, n + 2, period), node_f32);
    double a = p2 - p0;
    double b = ((2.0 * p0 - 5.0 * p1) + 4.0 * p2) - p3;
    double c = ((3.0 * p1 - p0) - 3.0 * p2) + p3;
    return -0.5 * ((a + 2.0 * b * d) + 3.0 * c * d * d);
}

static double pinning_force(int kind, uint64_t seed, uint32_t s, int64_t i, double u, int64_t period)
{
    return pinning_force_nodes(kind, seed, s, i, u, period, 0);
}

/* The RB potential itself, V(i, u), for the spline pins: Catmull-Rom (RB, RB-G cubic) or
   linear (RB-G linear). */
static double rb_potential(int kind, uint64_t seed, uint32_t s, int64_t i, double u, int64_t period)
{
    double fl = floor(u);
    int64_t n = (int64_t)fl;
    double d = u - fl;
    if (kind == QO_RBG_LINEAR)
        return (1.0 - d) * rbg_value(seed, s, i, wrap_node(n, period)) + d * rbg_value(seed, s, i, wrap_node(n + 1, period));
    double p0 = potential_value(kind, seed, s, i, n - 1, period);
    double p1 = potential_value(kind, seed, s, i, n, period);
    double p2 = potential_value(kind, seed, s, i, n + 1, period);
    double p3 = potential_value(kind, seed, s, i, n + 2, period);
    double a = p2 - p0;
    double b = ((2.0 * p0 - 5.0 * p1) + 4.0 * p2) - p3;
    double c = ((3.0 * p1 - p0) - 3.0 * p2) + p3;
    return 0.5 * (((2.0 * p1 + a * d) + b * d * d) + c * d * d * d);
}

void oracle_disorder_values(int kind, uint64_t seed, uint32_t s, const int64_t* i, const int64_t* n,
                            int64_t count, double* out, int64_t period)
{
    for (int64_t k = 0; k < count; ++k) {
        int64_t m = wrap_node(n[k], period);
        out[k] = (kind == QO_RF) ? rf_value(seed, s, i[k], m)
                 : (kind == QO_RB) ? rb_value(seed, s, i[k], m)
                                   : rbg_value(seed, s, i[k], m);
    }
}

void oracle_pinning_force(int kind, uint64_t seed, uint32_t s, const int64_t* i, const double* u,
                          int64_t count, double* out, int64_t period)
{
    for (int64_t k = 0; k < count; ++k)
        out[k] = pinning_force(kind, seed, s, i[k], u[k], period);
}

void oracle_rb_potential(int kind, uint64_t seed, uint32_t s, const int64_t* i, const double* u, int64_t count,
                         double* out, int64_t period)
{
    for (int64_t k = 0; k < count; ++k)
        out[k] = rb_potential(kind, seed, s, i[k], u[k], period);
}

/* ------------------------------------------------------------------------------------ */
/* Compensated (Neumaier) summation for the observables.                                */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    double s, c;
} nsum_t;

static void nsum_add(nsum_t* a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static double nsum_value(const nsum_t* a) { return a->s + a->c; }

/* Observables of one chain at the current state: v (Eq. 3 per sample, from the forces F
   at this state), ubar (Eq. 4) and w2 (Eq. 5, two-pass). */
static void observe(int64_t L, double f, const double* u, const double* F, double* v, double* ubar,
                    double* w2)
{
    nsum_t sf = {0, 0}, su = {0, 0}, sq = {0, 0};
    for (int64_t i = 0; i < L; ++i) {
        nsum_add(&sf, F[i]);
        nsum_add(&su, u[i]);
    }
    double mean = nsum_value(&su) / (double)L;
    for (int64_t i = 0; i < L; ++i) {
        double e = u[i] - mean;
        nsum_add(&sq, e * e);
    }
    *v = f + nsum_value(&sf) / (double)L;
    *ubar = mean;
    *w2 = nsum_value(&sq) / (double)L;
}

/* ------------------------------------------------------------------------------------ */
/* One chain: Euler steps with observations at the listed step counts.                  */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    int64_t L;
    uint32_t s;
    double f, dt;
    int kind;
    uint64_t seed;
    int64_t period;        /* disorder period M in u (0: aperiodic) */
    int node_f32;          /* 1: disorder values rounded to FP32 (the FP32 node model) */
    const double* u0;      /* initial state [L] or NULL for the flat start */
    const int64_t* steps;  /* observation steps, strictly increasing, >= 0 */
    int32_t n_times;
    double* v_out;         /* [n_times] (stride 'stride') or NULL */
    double* ubar_out;
    double* w2_out;
    int64_t stride;
    double* u_final;       /* [L] or NULL: state after the last observation step */
    int status;
} chain_job_t;

static int run_chain(chain_job_t* job)
{
    const int64_t L = job->L;
    double* u = (double*)malloc((size_t)L * sizeof(double));
    double* un = (double*)malloc((size_t)L * sizeof(double));
    double* F = (double*)malloc((size_t)L * sizeof(double));
    if (!u || !un || !F) {
        free(u); free(un); free(F);
        return -2;
    }
    for (int64_t i = 0; i < L; ++i)
        u[i] = job->u0 ? job->u0[i] : 0.0;
    int64_t step = 0;
    for (int32_t k = 0; k < job->n_times; ++k) {
        int64_t target = job->steps[k];
        for (;;) {
            for (int64_t i = 0; i < L; ++i)
                F[i] = pinning_force_nodes(job->kind, job->seed, job->s, i, u[i], job->period, job->node_f32);
            if (step == target)
                break;
            for (int64_t i = 0; i < L; ++i) {
                int64_t ip = (i + 1 == L) ? 0 : i + 1;
                int64_t im = (i == 0) ? L - 1 : i - 1;
                double lap = (u[ip] + u[im]) - 2.0 * u[i];
                un[i] = u[i] + job->dt * ((lap + job->f) + F[i]);
            }
            double* t = u; u = un; un = t;
            ++step;
        }
        double v, ub, w2;
        observe(L, job->f, u, F, &v, &ub, &w2);
        if (job->v_out) job->v_out[k * job->stride] = v;
        if (job->ubar_out) job->ubar_out[k * job->stride] = ub;
        if (job->w2_out) job->w2_out[k * job->stride] = w2;
    }
    if (job->u_final)
        memcpy(job->u_final, u, (size_t)L * sizeof(double));
    free(u); free(un); free(F);
    return 0;
}

typedef struct {
    chain_job_t* jobs;
    int32_t n_jobs;
    int32_t next;
    pthread_mutex_t lock;
} pool_t;

static void* pool_worker(void* arg)
{
    pool_t* p = (pool_t*)arg;
    for (;;) {
        pthread_mutex_lock(&p->lock);
        int32_t j = p->next++;
        pthread_mutex_unlock(&p->lock);
        if (j >= p->n_jobs)
            return NULL;
        p->jobs[j].status = run_chain(&p->jobs[j]);
    }
}

static int run_jobs(chain_job_t* jobs, int32_t n_jobs, int32_t n_threads)
{
    if (n_threads <= 0) {
        long c = sysconf(_SC_NPROCESSORS_ONLN);
        n_threads = c > 0 ? (int32_t)c : 1;
    }
    if (n_threads > n_jobs)
        n_threads = n_jobs;
    pool_t pool;
    pool.jobs = jobs;
    pool.n_jobs = n_jobs;
    pool.next = 0;
    pthread_mutex_init(&pool.lock, NULL);
    pthread_t* th = (pthread_t*)malloc((size_t)n_threads * sizeof(pthread_t));
    if (!th)
        return -2;
    int32_t started = 0;
    for (int32_t t = 1; t < n_threads; ++t) {
        if (pthread_create(&th[started], NULL, pool_worker, &pool) != 0)
            break;
        ++started;
    }
    pool_worker(&pool);
    for (int32_t t = 0; t < started; ++t)
        pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&pool.lock);
    for (int32_t j = 0; j < n_jobs; ++j)
        if (jobs[j].status != 0)
            return jobs[j].status;
    return 0;
}

/*
 * Run n_chains independent chains; chain c has length L[c], sample index s[c], drive f[c]
 * and disorder kind kind[c]; the disorder is periodic in u with period `period` (0:
 * aperiodic).  Observations at steps[0..n_times) are written to
 * v_out/ubar_out/w2_out[k * n_chains + c].  u0 (optional) and u_final (optional) hold the
 * chains one after another (chain c starts at offset sum_{c'<c} L[c']).  node_f32 = 1 runs
 * the FP32 node model (disorder values rounded to FP32); 0 the exact dynamics.
 * Returns 0, or -1 on bad arguments, -2 on allocation failure.
 */
int oracle_run(int32_t n_chains, const int64_t* L, const uint32_t* s, const double* f, const int32_t* kind,
               double dt, uint64_t seed, const double* u0, const int64_t* steps, int32_t n_times,
               double* v_out, double* ubar_out, double* w2_out, double* u_final, int32_t n_threads,
               int64_t period, int32_t node_f32)
{
    if (n_chains < 1 || n_times < 0)
        return -1;
    for (int32_t k = 0; k < n_times; ++k)
        if (steps[k] < 0 || (k > 0 && steps[k] <= steps[k - 1]))
            return -1;
    chain_job_t* jobs = (chain_job_t*)calloc((size_t)n_chains, sizeof(chain_job_t));
    if (!jobs)
        return -2;
    int64_t off = 0;
    for (int32_t c = 0; c < n_chains; ++c) {
        if (L[c] < 1) {
            free(jobs);
            return -1;
        }
        jobs[c].L = L[c];
        jobs[c].s = s[c];
        jobs[c].f = f[c];
        jobs[c].dt = dt;
        jobs[c].kind = kind[c];
        jobs[c].seed = seed;
        jobs[c].period = period;
        jobs[c].node_f32 = node_f32 != 0;
        jobs[c].u0 = u0 ? u0 + off : NULL;
        jobs[c].steps = steps;
        jobs[c].n_times = n_times;
        jobs[c].v_out = v_out ? v_out + c : NULL;
        jobs[c].ubar_out = ubar_out ? ubar_out + c : NULL;
        jobs[c].w2_out = w2_out ? w2_out + c : NULL;
        jobs[c].stride = n_chains;
        jobs[c].u_final = u_final ? u_final + off : NULL;
        off += L[c];
    }
    int rc = run_jobs(jobs, n_chains, n_threads);
    free(jobs);
    return rc;
}

/*
 * Light-cone evaluation: after n_steps Euler steps from the flat start, site i depends only
 * on sites i - n_steps .. i + n_steps (the stencil has radius 1).  This evaluates sites
 * i0 .. i0 + w - 1 (indices mod L) of chain s exactly as the periodic run would, from a
 * window of w + 2 n_steps sites; requires w + 2 n_steps <= L so that no site of the window
 * is used twice.  Writes u after n_steps to u_out[0..w) and, if F_out is given, the pinning
 * force at that state.  Returns 0, -1 on bad arguments, -2 on allocation failure.
 */
int oracle_lightcone(int64_t L, uint32_t s, double f, double dt, int kind, uint64_t seed, int64_t i0,
                     int64_t w, int64_t n_steps, double* u_out, double* F_out, int64_t period)
{
    if (L < 1 || w < 1 || n_steps < 0 || w + 2 * n_steps > L)
        return -1;
    int64_t W = w + 2 * n_steps;
    double* u = (double*)calloc((size_t)W, sizeof(double));
    double* un = (double*)calloc((size_t)W, sizeof(double));
    double* F = (double*)calloc((size_t)W, sizeof(double));
    int64_t* gi = (int64_t*)malloc((size_t)W * sizeof(int64_t));
    if (!u || !un || !F || !gi) {
        free(u); free(un); free(F); free(gi);
        return -2;
    }
    for (int64_t j = 0; j < W; ++j) {
        int64_t g = (i0 - n_steps + j) % L;
        gi[j] = g < 0 ? g + L : g;
    }
    for (int64_t k = 0; k < n_steps; ++k) {
        /* sites k .. W-1-k are exact before this step; k+1 .. W-2-k after it */
        for (int64_t j = k; j <= W - 1 - k; ++j)
            F[j] = pinning_force(kind, seed, s, gi[j], u[j], period);
        for (int64_t j = k + 1; j <= W - 2 - k; ++j) {
            double lap = (u[j + 1] + u[j - 1]) - 2.0 * u[j];
            un[j] = u[j] + dt * ((lap + f) + F[j]);
        }
        for (int64_t j = k + 1; j <= W - 2 - k; ++j)
            u[j] = un[j];
    }
    for (int64_t j = 0; j < w; ++j) {
        u_out[j] = u[n_steps + j];
        if (F_out)
            F_out[j] = pinning_force(kind, seed, s, gi[n_steps + j], u[n_steps + j], period);
    }
    free(u); free(un); free(F); free(gi);
    return 0;
}
