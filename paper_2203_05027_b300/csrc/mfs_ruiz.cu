// Ruiz equilibration of the problem data (host), a convergence variant outside the paper, whose
// Algorithm 1 runs on the data as given. D. Ruiz's scaling ("A scaling algorithm to equilibrate
// both rows and columns norms in matrices", 2001): each pass takes the infinity norms of the rows and
// of the columns of the current matrix over the listed entries (the columns of one Lorentz cone share
// the largest of their norms, so that the cone is scaled as one block and stays a cone) and divides
// every row and column by the square root of its norm (a zero norm leaves it alone). The solver then
// runs on A' = D A E, b' = D b, c' = E c; x = E x', z = E z', lambda = D lambda', delta = E^-1 delta'.
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mfs.h"

namespace {

thread_local std::string g_ruiz_error;

mfs_status ruiz_fail(const char* msg) {
    g_ruiz_error = msg;
    return MFS_ERR_INVALID;
}

}  // namespace

extern "C" {

const char* mfs_ruiz_last_error(void) {
    return g_ruiz_error.c_str();
}

mfs_status mfs_ruiz_scale(int64_t m, int64_t n, int64_t nnz, const int64_t* row, const int64_t* col, double* val,
                          double* b, double* c, int64_t ncones, const mfs_cone* cones, int32_t passes, double* d,
                          double* e) {
    g_ruiz_error.clear();
    if (m < 0 || n < 0 || nnz < 0 || ncones < 0 || passes < 0) return ruiz_fail("negative size or passes");
    if ((nnz > 0 && (!row || !col || !val)) || (m > 0 && (!b || !d)) || (n > 0 && (!c || !e)) ||
        (ncones > 0 && !cones))
        return ruiz_fail("NULL array");
    for (int64_t k = 0; k < nnz; ++k) {
        if (row[k] < 0 || row[k] >= m || col[k] < 0 || col[k] >= n) return ruiz_fail("index out of range");
        if (!std::isfinite(val[k])) return ruiz_fail("non-finite value");
    }
    // the column blocks that share one factor: the Lorentz cones of more than one column
    std::vector<std::pair<int64_t, int64_t>> blocks;
    int64_t off = 0;
    for (int64_t q = 0; q < ncones; ++q) {
        if (cones[q].size < 1) return ruiz_fail("cone of size < 1");
        if (cones[q].kind != MFS_CONE_NONNEG && cones[q].kind != MFS_CONE_SOC) return ruiz_fail("unknown cone kind");
        if (cones[q].kind == MFS_CONE_SOC && cones[q].size > 1) blocks.push_back({off, off + cones[q].size});
        off += cones[q].size;
    }
    if (off != n) return ruiz_fail("cone sizes must sum to n");
    for (int64_t i = 0; i < m; ++i) d[i] = 1.0;
    for (int64_t j = 0; j < n; ++j) e[j] = 1.0;
    std::vector<double> r((size_t)m), q((size_t)n), sr((size_t)m), sc((size_t)n);
    for (int32_t p = 0; p < passes; ++p) {
        std::fill(r.begin(), r.end(), 0.0);
        std::fill(q.begin(), q.end(), 0.0);
        for (int64_t k = 0; k < nnz; ++k) {
            const double a = std::fabs(val[k]);
            if (a > r[(size_t)row[k]]) r[(size_t)row[k]] = a;
            if (a > q[(size_t)col[k]]) q[(size_t)col[k]] = a;
        }
        for (const auto& bl : blocks) {
            double mx = 0.0;
            for (int64_t j = bl.first; j < bl.second; ++j) mx = q[(size_t)j] > mx ? q[(size_t)j] : mx;
            for (int64_t j = bl.first; j < bl.second; ++j) q[(size_t)j] = mx;
        }
        for (int64_t i = 0; i < m; ++i) sr[(size_t)i] = r[(size_t)i] > 0.0 ? 1.0 / std::sqrt(r[(size_t)i]) : 1.0;
        for (int64_t j = 0; j < n; ++j) sc[(size_t)j] = q[(size_t)j] > 0.0 ? 1.0 / std::sqrt(q[(size_t)j]) : 1.0;
        for (int64_t k = 0; k < nnz; ++k) val[k] = val[k] * sr[(size_t)row[k]] * sc[(size_t)col[k]];
        for (int64_t i = 0; i < m; ++i) d[i] *= sr[(size_t)i];
        for (int64_t j = 0; j < n; ++j) e[j] *= sc[(size_t)j];
    }
    for (int64_t i = 0; i < m; ++i) b[i] *= d[i];
    for (int64_t j = 0; j < n; ++j) c[j] *= e[j];
    return MFS_OK;
}

mfs_status mfs_ruiz_unscale(int64_t m, int64_t n, const double* d, const double* e, double* x, double* lambda,
                            double* z, double* delta) {
    if (m < 0 || n < 0 || (m > 0 && !d) || (n > 0 && !e)) return ruiz_fail("bad sizes or NULL factors");
    for (int64_t j = 0; j < n; ++j) {
        if (x) x[j] *= e[j];
        if (z) z[j] *= e[j];
        if (delta) delta[j] /= e[j];
    }
    if (lambda)
        for (int64_t i = 0; i < m; ++i) lambda[i] *= d[i];
    return MFS_OK;
}

mfs_status mfs_ruiz_scale_start(int64_t m, int64_t n, const double* d, const double* e, double* x, double* lambda,
                                double* z, double* delta) {
    if (m < 0 || n < 0 || (m > 0 && !d) || (n > 0 && !e)) return ruiz_fail("bad sizes or NULL factors");
    for (int64_t j = 0; j < n; ++j) {
        if (x) x[j] /= e[j];
        if (z) z[j] /= e[j];
        if (delta) delta[j] *= e[j];
    }
    if (lambda)
        for (int64_t i = 0; i < m; ++i) lambda[i] /= d[i];
    return MFS_OK;
}

}  // extern "C"
