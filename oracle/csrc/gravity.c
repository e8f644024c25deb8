/* CPU oracle helper (test infrastructure): reference gravity by direct
 * summation over tet point masses, g(x_i) = -G sum_k m_k (x_i - r_k) /
 * |x_i - r_k|^3 (paper Sec. 5.1, Newtonian kernel), parallel over targets.
 * src holds (r_x, r_y, r_z, m) per tet. */
#include <math.h>
#include <stdint.h>

void oracle_gravity_direct(int64_t nx, const double* x, int64_t ns, const double* src, double G, double* g) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nx; ++i) {
        double a0 = 0, a1 = 0, a2 = 0;
        const double x0 = x[3 * i], x1 = x[3 * i + 1], x2 = x[3 * i + 2];
        for (int64_t k = 0; k < ns; ++k) {
            const double d0 = x0 - src[4 * k], d1 = x1 - src[4 * k + 1], d2 = x2 - src[4 * k + 2];
            const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
            const double w = src[4 * k + 3] / (r2 * sqrt(r2));
            a0 += w * d0;
            a1 += w * d1;
            a2 += w * d2;
        }
        g[3 * i] = -G * a0;
        g[3 * i + 1] = -G * a1;
        g[3 * i + 2] = -G * a2;
    }
}
