// Checks mfs::host::static_resid_args_ok, the host-side argument rule of mfs_row_residuals_static:
// the row limit of the static scratch (at and one past it), negative sizes, the column limit, and a
// NULL in each array the sizes require, with the same arrays optional where a size is zero. Exit
// status 0 = pass.
#include <cstdio>

#include "mfs_host.h"

int main() {
    using mfs::host::static_resid_args_ok;
    const int64_t lim = 4194304;
    int bad = 0;
    auto expect = [&](bool got, bool want, const char* what) {
        if (got != want) {
            std::printf("FAIL: %s: got %d, want %d\n", what, (int)got, (int)want);
            bad = 1;
        }
    };
    const bool T = true, F = false;
    expect(static_resid_args_ok(lim, 10, lim, T, T, T, T, T, T, T), true, "m at the limit");
    expect(static_resid_args_ok(lim + 1, 10, lim, T, T, T, T, T, T, T), false, "m one past the limit");
    expect(static_resid_args_ok(INT64_MAX, 10, lim, T, T, T, T, T, T, T), false, "huge m");
    expect(static_resid_args_ok(-1, 10, lim, T, T, T, T, T, T, T), false, "negative m");
    expect(static_resid_args_ok(5, -1, lim, T, T, T, T, T, T, T), false, "negative n");
    expect(static_resid_args_ok(5, INT32_MAX, lim, T, T, T, T, T, T, T), false, "n = 2^31 - 1");
    expect(static_resid_args_ok(5, INT32_MAX - 1, lim, T, T, T, T, T, T, T), true, "n = 2^31 - 2");
    expect(static_resid_args_ok(5, 7, lim, T, T, T, T, T, T, F), false, "no out");
    expect(static_resid_args_ok(0, 0, lim, F, F, F, F, F, F, F), false, "no out, empty problem");
    expect(static_resid_args_ok(0, 0, lim, F, F, F, F, F, F, T), true, "empty problem");
    expect(static_resid_args_ok(0, 7, lim, F, F, F, F, T, F, T), true, "no rows: CSR, b, lambda optional");
    expect(static_resid_args_ok(0, 7, lim, F, F, F, F, F, F, T), false, "no rows but columns: x needed");
    expect(static_resid_args_ok(3, 0, lim, T, T, T, T, F, T, T), true, "no columns: x optional");
    const char* names[] = {"row_ptr", "col_idx", "val", "b", "x", "lambda"};
    for (int q = 0; q < 6; ++q) {
        bool h[6] = {T, T, T, T, T, T};
        h[q] = F;
        expect(static_resid_args_ok(3, 7, lim, h[0], h[1], h[2], h[3], h[4], h[5], T), false, names[q]);
    }
    if (!bad) std::printf("ok\n");
    return bad;
}
