// FP64 geometry of the precalculation module (§3.3), shared by the FP32
// sparse tables and the BF16 tensor-core operands so both hold the same
// weights.  Stencil frame and configuration index as described in
// geometry.cu.
#pragma once

#include <math.h>

namespace cd {

// Length of {p + s u : s >= 0} inside the cube [lo, lo + 1]^3 (slab method).
__device__ __forceinline__ double path_in_cube(const double *p, const double *u, double lx, double ly, double lz)
{
    const double lo[3] = {lx, ly, lz};
    double enter = 0.0, leave = 1e300;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (u[a] == 0.0) {
            if (p[a] < lo[a] || p[a] > lo[a] + 1.0) return 0.0;
        } else {
            double s0 = (lo[a] - p[a]) / u[a];
            double s1 = (lo[a] + 1.0 - p[a]) / u[a];
            if (s0 > s1) {
                const double x = s0;
                s0 = s1;
                s1 = x;
            }
            enter = fmax(enter, s0);
            leave = fmin(leave, s1);
        }
    }
    return leave > enter ? leave - enter : 0.0;
}

// K_t[cfg][s] for direction u, in units of the shell's cell size: the path of
// the ray from the centre of the receiving cell A_k (k = l + t - 1) through
// stencil cell s = a + 6 b + 36 c, zero inside the inner region.
__device__ __forceinline__ double shell_weight(int t, int cfg, int s, const double *u)
{
    double p[3];
    int top[3];
    for (int a = 0; a < 3; ++a) {
        double x = 2.0;
        for (int j = 0; j < t; ++j) {
            const int o = (cfg >> (3 * (t - 1 - j))) & 7;
            x += (double)((o >> a) & 1) * ldexp(1.0, -j);
        }
        p[a] = x + ldexp(1.0, -t);
        top[a] = 2 + (((cfg >> (3 * (t - 1))) >> a) & 1);
    }
    const int a = s % 6, b = (s / 6) % 6, c = s / 36;
    const bool inner = (t == 1) ? (a == top[0] && b == top[1] && c == top[2])
                                : (abs(a - top[0]) <= 1 && abs(b - top[1]) <= 1 && abs(c - top[2]) <= 1);
    return inner ? 0.0 : path_in_cube(p, u, a, b, c);
}

// shell_weight averaged over the ns rays u[0 .. 3 ns - 1] of one direction
// (ns = 1: the direction itself, bit for bit)
__device__ __forceinline__ double shell_weight_avg(int t, int cfg, int s, const double *u, int ns)
{
    double acc = 0.0;
    for (int j = 0; j < ns; ++j) acc += shell_weight(t, cfg, s, u + 3 * j);
    return acc / ns;
}

}  // namespace cd
