// mfs_measures.h -- the stopping-rule measures of a residual record (host side, shared by the
// single, batched and shared-A solvers).
#pragma once

#include <algorithm>
#include <cmath>

#include "../../include/mfs.h"

namespace mfs {

// Largest |entry| of w - P(w) for one Lorentz cone, from w_1 and alpha = ||w_{2..}||: |w_1| when w
// lies in the polar cone (then |w_1| >= alpha >= every |w_t|), 0 inside the cone, else
// (alpha - w_1)/2, the head's entry, since the tail's entries w_t (alpha - w_1)/(2 alpha) are no
// larger.
#ifdef __CUDACC__
__host__ __device__
#endif
inline double lorentz_distinf(double w1, double alpha) {
    if (alpha <= -w1) return std::fabs(w1);
    if (alpha <= w1) return 0.0;
    return 0.5 * (alpha - w1);
}

// r_scs and r_osqp of mfs_residuals_t from its norms: the paper's l2 rule against SCS and
// infinity-norm rule against OSQP (Sec. V), with the cone constraint x in K joining the primal
// rows and the cone multiplier taken out of the dual residual; q = eps_rel / eps_abs of the OSQP
// rule. NaN in any part gives NaN.
inline void stop_measures(mfs_residuals_t* r, double q) {
    const double p2 = std::sqrt(r->nrm_res_p * r->nrm_res_p + r->nrm_xdist * r->nrm_xdist) / (1.0 + r->nrm_b);
    const double d2 = r->nrm_sdist / (1.0 + r->nrm_c);
    r->r_scs = std::max(std::max(p2, d2), r->r_gap);
    const double pi = std::max(r->inf_res_p, r->inf_xdist) / (1.0 + q * std::max(std::max(r->inf_ax, r->inf_x), r->inf_b));
    const double di = r->inf_sdist / (1.0 + q * std::max(r->inf_atl, r->inf_c));
    r->r_osqp = std::max(pi, di);
    if (std::isnan(p2) || std::isnan(d2) || std::isnan(r->r_gap)) r->r_scs = NAN;
    if (std::isnan(pi) || std::isnan(di)) r->r_osqp = NAN;
}

}  // namespace mfs
