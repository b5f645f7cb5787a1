// Dense bounded-variable primal simplex (host, FP64) for the small linear
// programs of the allocation repair: choose convex weights of a few jobs'
// optimal allocations so that the total usage meets the resource limits
// (the paper's Section 3 says any optimal allocation solves every job's
// subproblem at optimal prices; which ones to mix is left open).
//
//     minimize c^T x   subject to   A x = b,   0 <= x <= ub   (ub may be +inf)
//
// The caller gives a starting basis of unit columns: for every row r one
// column whose entries are 1 in row r and 0 elsewhere, with b >= 0, so that
// x_B = b is feasible.  After a first solve the cost vector and upper bounds
// may be changed (keeping the current point feasible) and the solve resumed:
// this is how a two-phase (feasibility, then objective) solve is run.
#pragma once

#include <vector>

namespace ra {
namespace lp {

enum Result { kOptimal = 0, kIterLimit = 1, kUnbounded = 2, kBadStart = 3 };

class Simplex {
public:
    // A is row-major rows x cols; basis[r] is the unit column of row r.
    Simplex(int rows, int cols, std::vector<double> A, std::vector<double> b,
            std::vector<double> c, std::vector<double> ub, std::vector<int> basis);

    Result solve(int max_iter);
    void set_cost(const std::vector<double> &c) { c_ = c; }
    // New upper bound of column j; the current value of x_j must not exceed it.
    void set_upper(int j, double ub) { ub_[j] = ub; }
    std::vector<double> x() const;
    double objective() const;
    int iterations() const { return iters_; }

private:
    int rows_, cols_;
    std::vector<double> T_;      // tableau B^-1 A, rows x cols
    std::vector<double> beta_;   // values of the basic variables
    std::vector<double> c_, ub_;
    std::vector<int> basis_;     // basic column of each row
    std::vector<int> pos_;       // row of a basic column, -1 if nonbasic
    std::vector<char> at_upper_; // nonbasic column at its upper bound
    int iters_ = 0;
    bool ok_ = true;

    double &t(int r, int j) { return T_[static_cast<size_t>(r) * cols_ + j]; }
    double t(int r, int j) const { return T_[static_cast<size_t>(r) * cols_ + j]; }
    void pivot(int r, int j);
};

}  // namespace lp
}  // namespace ra
