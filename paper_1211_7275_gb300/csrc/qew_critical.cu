// qew_critical.cu -- exact critical force of a periodic random-field sample (host code).
//
// Sec. III.B of arXiv:1211.7275 defines, for a sample periodic in u with period M (the L x M
// system), the critical force f_c^s as the largest drive at which a pinned configuration exists,
// and the critical configuration as that pinned configuration; the paper computes both with an
// exact algorithm built on Middleton's theorems (it cites it, Sec. III.B and Sec. IV.A).  This file
// computes them for the random-field disorder with linear interpolation (Case 4), without following
// the dynamics to convergence near the threshold:
//
//   With every site's cell n_i fixed, the pinning force is linear in the offset d_i = u_i - n_i,
//   F_i = R_i(n_i) + s_i d_i with s_i = R_i(n_i + 1) - R_i(n_i), so the static equation
//   lap(u) + f + F(u) = 0 is the linear system
//       M d = f + R(n) + lap(n),   M = -lap - diag(s)          (periodic, symmetric, tridiagonal).
//   A static solution is stable (a pinned configuration) when M is positive definite; then M is a
//   nonsingular M-matrix, so w = dd/df = M^-1 1 > 0 and the whole line moves forward as f grows
//   (no-passing).  Along such a branch the configuration is exactly d(f) = d + (f - f_0) w, until
//   the first site reaches its cell's upper edge, at f + (1 - d_k) / w_k.  There the force is
//   continuous, so the configuration is unchanged; the site's cell advances, M changes in one
//   diagonal entry, and either the new M is positive definite (the branch goes on) or the pinned
//   configuration has reached the end of its branch (a saddle-node) and the line depins locally: an
//   avalanche at fixed f.  The avalanche is followed with the Euler map (monotone forward from a
//   pinned configuration, Middleton's no-passing) until the line pins again, and the branch
//   following resumes from the new pinned configuration; or until every site has advanced by M, in
//   which case the motion repeats one period higher forever and f is the critical force: the last
//   pinned configuration before that avalanche is the critical configuration.
//
// Everything is FP64.  The pinned branches are computed exactly (up to rounding); only the
// avalanches use the dynamics, away from the threshold's critical slowing down.
#include <cmath>
#include <cstdint>
#include <new>
#include <string>
#include <vector>

#include "qew.h"
#include "qew_internal.h"

namespace {

struct Sample {
    int64_t L, M;
    const double* R;   // [L][M]: R(i, m), m = n mod M
    double r(int64_t i, int64_t n) const
    {
        int64_t m = n % M;
        if (m < 0)
            m += M;
        return R[i * M + m];
    }
};

// Solve M x = rhs for the periodic tridiagonal M with diagonal dg[i] and every neighbour coupling
// -1 (site 0 couples to sites 1 and L - 1; for L = 2 the two couplings add).  Eliminates the open
// chain 1 .. L-1 (Thomas algorithm) and then site 0 through its Schur complement.  Returns false
// when M is not positive definite (a non-positive pivot or Schur complement).
bool solve_periodic(int64_t L, const std::vector<double>& dg, const std::vector<double>& rhs,
                    std::vector<double>& x, std::vector<double>& p, std::vector<double>& y1,
                    std::vector<double>& y2)
{
    if (L == 1) {
        // the site is its own neighbour on both sides: the Laplacian vanishes, M = dg[0] - 2
        const double m = dg[0] - 2.0;
        if (!(m > 0.0))
            return false;
        x[0] = rhs[0] / m;
        return true;
    }
    const int64_t n = L - 1;   // chain sites 1 .. L-1 at positions 0 .. n-1
    // c: coupling of site 0 to the chain (-1 to site 1, -1 to site L-1)
    // forward elimination of T (diag dg[1..L-1], off-diagonal -1) on both right-hand sides
    for (int64_t k = 0; k < n; ++k) {
        const int64_t i = k + 1;
        double piv = dg[i];
        double a1 = rhs[i];
        double a2 = 0.0;
        if (k == 0)
            a2 -= 1.0;
        if (k == n - 1)
            a2 -= 1.0;
        if (k > 0) {
            piv -= 1.0 / p[k - 1];
            a1 += y1[k - 1] / p[k - 1];
            a2 += y2[k - 1] / p[k - 1];
        }
        if (!(piv > 0.0))
            return false;
        p[k] = piv;
        y1[k] = a1;
        y2[k] = a2;
    }
    // back substitution: z = T^-1 (.) in place
    for (int64_t k = n - 1; k >= 0; --k) {
        double z1 = y1[k], z2 = y2[k];
        if (k + 1 < n) {
            z1 += y1[k + 1];
            z2 += y2[k + 1];
        }
        y1[k] = z1 / p[k];
        y2[k] = z2 / p[k];
    }
    // c^T z: c has -1 at chain positions 0 and n - 1 (the same position twice for L = 2)
    const double cz1 = -y1[0] - y1[n - 1];
    const double cz2 = -y2[0] - y2[n - 1];
    const double schur = dg[0] - cz2;
    if (!(schur > 0.0))
        return false;
    x[0] = (rhs[0] - cz1) / schur;
    for (int64_t k = 0; k < n; ++k)
        x[k + 1] = y1[k] - x[0] * y2[k];
    return true;
}

struct Solver {
    Sample smp;
    double dt;
    std::vector<int64_t> n;    // cells
    std::vector<double> d;     // offsets u - n
    std::vector<double> dg, rhs, w, ones, p, y1, y2;
    int64_t events = 0, dyn_steps = 0;

    explicit Solver(const Sample& s, double dt_) : smp(s), dt(dt_)
    {
        const size_t L = static_cast<size_t>(s.L);
        n.assign(L, 0);
        d.assign(L, 0.0);
        dg.resize(L);
        rhs.resize(L);
        w.resize(L);
        ones.assign(L, 1.0);
        p.resize(L);
        y1.resize(L);
        y2.resize(L);
    }

    int64_t nb(int64_t i, int dir) const
    {
        const int64_t L = smp.L;
        return dir > 0 ? (i + 1 == L ? 0 : i + 1) : (i == 0 ? L - 1 : i - 1);
    }

    // the linear system of the current cells at drive f: diagonal and right-hand side
    void assemble(double f)
    {
        const int64_t L = smp.L;
        for (int64_t i = 0; i < L; ++i) {
            const double r0 = smp.r(i, n[i]);
            const double s = smp.r(i, n[i] + 1) - r0;
            dg[i] = 2.0 - s;
            const double lapn = static_cast<double>(n[nb(i, 1)] - n[i]) + static_cast<double>(n[nb(i, -1)] - n[i]);
            rhs[i] = (f + r0) + lapn;
        }
    }

    // exact static offsets for the current cells at f; false if not stable
    bool static_solution(double f)
    {
        assemble(f);
        return solve_periodic(smp.L, dg, rhs, d, p, y1, y2);
    }

    // Euler relaxation at fixed f from (n, d) until pinned (max |velocity| < v_tol) or runaway:
    // every site within 1e-4 of M past its position in (ref_n, ref_d) or beyond.  At f_c^s itself
    // the avalanche from the end of the critical branch ends on the critical configuration shifted
    // by one period (a marginal fixed point it approaches without reaching), so the margin is what
    // decides there; below f_c^s the line pins well short of a period.  The state is kept split into
    // integer cells and offsets, so the velocities keep their precision at any height of the line.
    // Returns 1 pinned, 2 runaway, 0 undecided.
    int relax(double f, double v_tol, int64_t max_steps, const std::vector<int64_t>& ref_n,
              const std::vector<double>& ref_d)
    {
        const int64_t L = smp.L;
        std::vector<double> dn(L);
        int result = 0;
        for (int64_t step = 0; step < max_steps; ++step) {
            double vmax = 0.0;
            for (int64_t i = 0; i < L; ++i) {
                const int64_t ip = nb(i, 1), im = nb(i, -1);
                const double lap = static_cast<double>((n[ip] - n[i]) + (n[im] - n[i])) + ((d[ip] + d[im]) - 2.0 * d[i]);
                const double v = (lap + f) + ((1.0 - d[i]) * smp.r(i, n[i]) + d[i] * smp.r(i, n[i] + 1));
                vmax = std::fmax(vmax, std::fabs(v));
                dn[i] = d[i] + dt * v;
            }
            for (int64_t i = 0; i < L; ++i) {
                const double fl = std::floor(dn[i]);
                n[i] += static_cast<int64_t>(fl);
                d[i] = dn[i] - fl;
            }
            ++dyn_steps;
            if (vmax < v_tol) {
                result = 1;
                break;
            }
            if ((step & 63) == 63) {
                bool all = true;
                for (int64_t i = 0; i < L && all; ++i)
                    all = static_cast<double>(n[i] - ref_n[i]) + (d[i] - ref_d[i]) >= static_cast<double>(smp.M) - 1e-4;
                if (all) {
                    result = 2;
                    break;
                }
            }
        }
        return result;
    }

    // After a relaxation: the exact static solution of the cells it ended in, with sites that the
    // solve places just outside their cell moved into the neighbouring cell.  False if no stable
    // consistent assignment was found (the relaxation stopped near an unstable fixed point).
    bool polish(double f)
    {
        std::vector<int64_t> n_keep = n;
        std::vector<double> d_keep = d;
        for (int it = 0; it < 8; ++it) {
            if (!static_solution(f))
                break;
            bool moved = false;
            for (int64_t i = 0; i < smp.L; ++i) {
                if (d[i] < 0.0) {
                    n[i] -= 1;
                    d[i] += 1.0;
                    moved = true;
                } else if (d[i] >= 1.0) {
                    n[i] += 1;
                    d[i] -= 1.0;
                    moved = true;
                }
            }
            if (!moved)
                return true;
        }
        n = n_keep;
        d = d_keep;
        return false;
    }

    // Motion at fixed f from the current configuration (a fixed point whose branch has ended, or
    // the flat start): a small forward push sets off the unstable direction, then the Euler map runs
    // until the line pins again (1, the exact pinned configuration in n, d) or has advanced by a
    // full period everywhere (2).  0 if neither happens within the limits.
    int avalanche(double f, double v_tol, int64_t max_steps)
    {
        const int64_t L = smp.L;
        const std::vector<int64_t> ref_n = n;
        const std::vector<double> ref_d = d;
        for (int attempt = 0; attempt < 64; ++attempt) {
            for (int64_t i = 0; i < L; ++i) {
                d[i] += 1e-6;
                if (d[i] >= 1.0) {
                    d[i] -= 1.0;
                    n[i] += 1;
                }
            }
            const int st = relax(f, v_tol, max_steps, ref_n, ref_d);
            if (st != 1)
                return st;
            if (polish(f))
                return 1;
        }
        return 0;
    }
};

}  // namespace

extern "C" int qew_critical_force_rf(int64_t L, int64_t M, const double* R, double dt, double f_start,
                                     double* f_c_out, double* u_c_out, int64_t* events_out,
                                     int64_t* dyn_steps_out)
{
    // M = 1 would make every site's force constant in u: no stable pinned configuration exists
    if (L < 1 || M < 2 || !R || !f_c_out)
        return (qew::set_last_error("need L >= 1, M >= 2, R and f_c_out"), QEW_EINVAL);
    if (!(dt > 0.0 && dt < 0.5) || !std::isfinite(f_start))
        return (qew::set_last_error("dt must lie in (0, 0.5) and f_start must be finite"), QEW_EINVAL);
    try {
        Sample smp{L, M, R};
        Solver s(smp, dt);
        const double v_tol = 1e-12;
        const int64_t max_relax = 2'000'000'000 / (L + 1) + 1'000'000;
        // the pinned configuration of the flat line at f_start
        double f = f_start;
        if (s.avalanche(f, v_tol, max_relax) != 1)
            return (qew::set_last_error("the flat line does not pin at f_start"), QEW_ESTATE);
        std::vector<int64_t> n_crit = s.n;
        std::vector<double> d_crit = s.d;
        double f_crit = f;
        const int64_t max_events = 200'000'000 / (L + 1) + 1'000'000;
        bool done = false;
        for (int64_t ev = 0; ev < max_events && !done; ++ev) {
            // follow the pinned branch: w = M^-1 1 > 0, the first site to reach its cell's edge
            s.assemble(f);
            if (!solve_periodic(L, s.dg, s.ones, s.w, s.p, s.y1, s.y2))
                return (qew::set_last_error("lost the pinned branch (numerical)"), QEW_ESTATE);
            int64_t k = -1;
            double best = INFINITY;
            for (int64_t i = 0; i < L; ++i) {
                const double df = (1.0 - s.d[i]) / s.w[i];
                if (df < best) {
                    best = df;
                    k = i;
                }
            }
            f += best;
            for (int64_t i = 0; i < L; ++i)
                s.d[i] += best * s.w[i];
            n_crit = s.n;
            d_crit = s.d;
            f_crit = f;
            s.n[k] += 1;
            s.d[k] = 0.0;
            ++s.events;
            // the next branch, if it is stable; else an avalanche at this f
            const std::vector<double> d_keep = s.d;
            if (s.static_solution(f)) {
                bool ok = true;
                for (int64_t i = 0; i < L && ok; ++i)
                    ok = s.d[i] > -1e-9 && s.d[i] < 1.0 + 1e-9;
                if (ok) {
                    for (int64_t i = 0; i < L; ++i)
                        s.d[i] = std::fmin(std::fmax(s.d[i], 0.0), std::nextafter(1.0, 0.0));
                    continue;
                }
            }
            s.d = d_keep;
            const int st = s.avalanche(f, v_tol, max_relax);
            if (st == 2)
                done = true;   // runaway: f is the critical force, (n_crit, d_crit) the critical configuration
            else if (st != 1)
                return (qew::set_last_error("an avalanche did not end within the step limit"), QEW_ESTATE);
        }
        if (!done)
            return (qew::set_last_error("no runaway within the event limit"), QEW_ESTATE);
        *f_c_out = f_crit;
        if (u_c_out)
            for (int64_t i = 0; i < L; ++i)
                u_c_out[i] = static_cast<double>(n_crit[i]) + d_crit[i];
        if (events_out)
            *events_out = s.events;
        if (dyn_steps_out)
            *dyn_steps_out = s.dyn_steps;
        return QEW_OK;
    } catch (const std::bad_alloc&) {
        return (qew::set_last_error("host allocation failed"), QEW_ENOMEM);
    }
}
