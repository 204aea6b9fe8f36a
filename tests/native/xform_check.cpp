// Host check of the pair transforms' double-float arithmetic (bt_xform.cuh):
// on random rigid poses (translations up to ~0.9 m), every entry of
// T_j T_i^-1 must equal the FP64-formed entry rounded once to single
// precision (the double-float sum is within ~2^-44 of it), and T_i^-1 must be
// the FP64 inverse rounded once.  Prints one line; exit status 1 on a
// mismatch of the inverse.  Compiled by tests/test_xform_host.py.
#define __host__
#define __device__
#define __forceinline__ inline
#include <cmath>
using std::fma;
#include "bt_xform.cuh"
#include <cstdio>
#include <random>
int main()
{
    std::mt19937_64 g(1);
    std::uniform_real_distribution<double> U(-1, 1);
    long n = 0, diff = 0, ulp2 = 0;
    double maxrel = 0;
    for (int trial = 0; trial < 20000; ++trial) {
        double T[2][12];
        for (int p = 0; p < 2; ++p) {
            // random rotation via quaternion, translation ~0.5 m
            double q[4]; double s = 0;
            for (int k = 0; k < 4; ++k) { q[k] = U(g); s += q[k] * q[k]; }
            s = std::sqrt(s); for (int k = 0; k < 4; ++k) q[k] /= s;
            const double w = q[0], x = q[1], y = q[2], z = q[3];
            double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w),
                           2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w),
                           2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)};
            for (int r = 0; r < 3; ++r) { for (int c = 0; c < 3; ++c) T[p][r * 4 + c] = R[r * 3 + c]; T[p][r * 4 + 3] = 0.4 * U(g) + (r == 2 ? 0.5 : 0); }
        }
        float si[32], sj[32];
        for (int k = 0; k < 15; ++k) { bt::xf_split_entry(T[0], k, si); bt::xf_split_entry(T[1], k, sj); }
        double inv[12];
        for (int r = 0; r < 3; ++r) { for (int c = 0; c < 3; ++c) inv[r * 4 + c] = T[0][c * 4 + r]; inv[r * 4 + 3] = bt::xf_inv_translation(T[0], r); }
        for (int e = 0; e < 12; ++e) {
            const int r = e >> 2, c = e & 3;
            double v = fma(T[1][r * 4 + 2], inv[2 * 4 + c], fma(T[1][r * 4 + 1], inv[1 * 4 + c], T[1][r * 4 + 0] * inv[0 * 4 + c]));
            if (c == 3) v += T[1][r * 4 + 3];
            const float ref = (float)v, got = bt::xf_pair_entry(sj, si, e);
            ++n;
            if (ref != got) { ++diff; if (std::fabs((double)ref - got) > 1.5 * std::ldexp(1.0, std::ilogb(ref) - 23)) ++ulp2; }
            if (v != 0) maxrel = std::fmax(maxrel, std::fabs((double)got - v) / std::fabs(v));
            if (bt::xf_inv_entry(si, e) != (float)inv[e]) { printf("xinv mismatch\n"); return 1; }
        }
    }
    printf("entries %ld differ %ld beyond1ulp %ld maxrel %.3e\n", n, diff, ulp2, maxrel);
    return 0;
}
