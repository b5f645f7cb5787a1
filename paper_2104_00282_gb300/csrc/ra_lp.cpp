// Dense bounded-variable primal simplex (see ra_lp.h).  Textbook method:
// nonbasic columns sit at a bound (0 or ub); the entering column is the one
// with the most improving reduced cost (Bland's smallest index after a run of
// degenerate steps, which rules out cycling); the ratio test lets a basic
// variable hit either of its bounds or the entering column flip to its other
// bound without a pivot.

#include "ra_lp.h"

#include <cmath>
#include <limits>

namespace ra {
namespace lp {

Simplex::Simplex(int rows, int cols, std::vector<double> A, std::vector<double> b,
                 std::vector<double> c, std::vector<double> ub, std::vector<int> basis)
    : rows_(rows), cols_(cols), T_(std::move(A)), beta_(std::move(b)), c_(std::move(c)),
      ub_(std::move(ub)), basis_(std::move(basis)), pos_(cols > 0 ? cols : 0, -1),
      at_upper_(cols > 0 ? cols : 0, 0)
{
    if (rows < 0 || cols < 0 || T_.size() != static_cast<size_t>(rows) * cols ||
        beta_.size() != static_cast<size_t>(rows) || c_.size() != static_cast<size_t>(cols) ||
        ub_.size() != static_cast<size_t>(cols) || basis_.size() != static_cast<size_t>(rows)) {
        ok_ = false;
        return;
    }
    for (int r = 0; r < rows; ++r) {
        const int j = basis_[r];
        if (j < 0 || j >= cols || pos_[j] >= 0 || !(beta_[r] >= 0.0) || beta_[r] > ub_[j]) {
            ok_ = false;
            return;
        }
        for (int i = 0; i < rows; ++i)
            if (t(i, j) != (i == r ? 1.0 : 0.0)) {
                ok_ = false;
                return;
            }
        pos_[j] = r;
    }
    for (int j = 0; j < cols; ++j)
        if (!(ub_[j] >= 0.0)) ok_ = false;
}

void Simplex::pivot(int r, int j)
{
    double *tr = &T_[static_cast<size_t>(r) * cols_];
    const double p = tr[j];
    for (int k = 0; k < cols_; ++k) tr[k] /= p;
    tr[j] = 1.0;
    for (int i = 0; i < rows_; ++i) {
        if (i == r) continue;
        double *ti = &T_[static_cast<size_t>(i) * cols_];
        const double f = ti[j];
        if (f == 0.0) continue;
        for (int k = 0; k < cols_; ++k) ti[k] -= f * tr[k];
        ti[j] = 0.0;
    }
    pos_[basis_[r]] = -1;
    basis_[r] = j;
    pos_[j] = r;
}

Result Simplex::solve(int max_iter)
{
    if (!ok_) return kBadStart;
    const double inf = std::numeric_limits<double>::infinity();
    std::vector<double> d(cols_, 0.0);
    int degenerate = 0;
    for (int it = 0; it < max_iter; ++it) {
        double cmax = 0.0;
        for (int j = 0; j < cols_; ++j) cmax = std::fmax(cmax, std::fabs(c_[j]));
        for (int j = 0; j < cols_; ++j) {
            if (pos_[j] >= 0) {
                d[j] = 0.0;
                continue;
            }
            double v = c_[j];
            for (int r = 0; r < rows_; ++r) v -= c_[basis_[r]] * t(r, j);
            d[j] = v;
        }
        const double eps_d = 1e-11 * (1.0 + cmax);
        const bool bland = degenerate > 50;
        int jin = -1;
        double best = 0.0;
        for (int j = 0; j < cols_; ++j) {
            if (pos_[j] >= 0) continue;
            const bool elig = at_upper_[j] ? (d[j] > eps_d) : (d[j] < -eps_d && ub_[j] > 0.0);
            if (!elig) continue;
            if (bland) {
                jin = j;
                break;
            }
            if (std::fabs(d[j]) > best) {
                best = std::fabs(d[j]);
                jin = j;
            }
        }
        if (jin < 0) return kOptimal;
        const double dir = at_upper_[jin] ? -1.0 : 1.0;
        // ratio test: the entering value moves by dir * theta, basic r by -dir * T[r][jin] * theta
        double colmax = 0.0;
        for (int r = 0; r < rows_; ++r) colmax = std::fmax(colmax, std::fabs(t(r, jin)));
        const double eps_p = 1e-9 * colmax;
        double theta = ub_[jin];  // the entering column's own bound (a flip)
        int rout = -1;
        bool out_upper = false;
        for (int r = 0; r < rows_; ++r) {
            const double a = t(r, jin);
            if (std::fabs(a) <= eps_p) continue;
            const double rate = -dir * a;
            double lim;
            bool up;
            if (rate < 0.0) {
                lim = beta_[r] / -rate;
                up = false;
            } else {
                const double u = ub_[basis_[r]];
                if (!(u < inf)) continue;
                lim = (u - beta_[r]) / rate;
                up = true;
            }
            if (lim < 0.0) lim = 0.0;
            if (lim < theta || (lim == theta && rout >= 0 && std::fabs(a) > std::fabs(t(rout, jin)))) {
                theta = lim;
                rout = r;
                out_upper = up;
            }
        }
        if (!(theta < inf)) return kUnbounded;
        degenerate = theta > 0.0 ? 0 : degenerate + 1;
        for (int r = 0; r < rows_; ++r) {
            double v = beta_[r] - dir * t(r, jin) * theta;
            const double u = ub_[basis_[r]];
            if (v < 0.0) v = 0.0;  // rounding: basic variables stay within their bounds
            if (v > u) v = u;
            beta_[r] = v;
        }
        ++iters_;
        if (rout < 0) {
            at_upper_[jin] = at_upper_[jin] ? 0 : 1;
            continue;
        }
        const double vin = at_upper_[jin] ? ub_[jin] - theta : theta;
        const int jout = basis_[rout];
        pivot(rout, jin);
        beta_[rout] = vin;
        at_upper_[jin] = 0;
        at_upper_[jout] = out_upper ? 1 : 0;
    }
    return kIterLimit;
}

std::vector<double> Simplex::x() const
{
    std::vector<double> x(cols_, 0.0);
    for (int j = 0; j < cols_; ++j)
        x[j] = pos_[j] >= 0 ? beta_[pos_[j]] : (at_upper_[j] ? ub_[j] : 0.0);
    return x;
}

double Simplex::objective() const
{
    const std::vector<double> v = x();
    double s = 0.0;
    for (int j = 0; j < cols_; ++j) s += c_[j] * v[j];
    return s;
}

}  // namespace lp
}  // namespace ra

#ifdef RA_LP_TEST_EXPORT
// C entry for the CPU unit test of the simplex (built only into the test's
// own shared object, never into libra.so).
extern "C" int ra_lp_test_solve(int rows, int cols, const double *A, const double *b,
                                const double *c, const double *ub, const int *basis, int max_iter,
                                double *x, double *obj)
{
    ra::lp::Simplex s(rows, cols, std::vector<double>(A, A + static_cast<size_t>(rows) * cols),
                      std::vector<double>(b, b + rows), std::vector<double>(c, c + cols),
                      std::vector<double>(ub, ub + cols), std::vector<int>(basis, basis + rows));
    const ra::lp::Result r = s.solve(max_iter);
    const std::vector<double> v = s.x();
    for (int j = 0; j < cols; ++j) x[j] = v[j];
    *obj = s.objective();
    return static_cast<int>(r);
}
#endif
