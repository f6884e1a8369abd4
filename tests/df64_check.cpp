// Host check of the bit-level double-float conversions of df64.cuh (compiled by
// tests/test_host_df64.py with g++): x = hi + lo to 2^-46 relative for |x| >= 2^-80 (to
// 2^-126 absolute below), |lo| <= 2^-23 |hi|, hi never larger in magnitude than x, sign of lo
// = sign of x, float -> double widening exact.
#define __host__
#define __device__
#define __forceinline__ inline
#include "../paper_1701_08935_gb300/csrc/df64.cuh"

#include <cmath>
#include <cstdio>
#include <random>

int main() {
    std::mt19937_64 rng(12345);
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    int bad = 0;
    double worst = 0.0;
    for (int i = 0; i < 1000000; ++i) {
        double x = U(rng) * std::pow(10.0, (int)(rng() % 60) - 30);
        if (i % 101 == 0) x = 0.0;
        if (i % 103 == 0) x = -std::ldexp(1.0, (int)(rng() % 200) - 100);
        if (i % 107 == 0) x = std::nextafter(1.0, 2.0) * (rng() % 2 ? 1 : -1);
        float hi, lo;
        zolo::df_split(x, hi, lo);
        const double back = (double)hi + (double)lo;
        const double rel = x != 0.0 ? std::fabs(back - x) / std::fabs(x) : std::fabs(back);
        if (std::fabs(x) >= std::ldexp(1.0, -80)) worst = std::max(worst, rel);
        if (std::fabs(x) >= std::ldexp(1.0, -80) ? rel > std::ldexp(1.0, -46)
                                                 : std::fabs(back - x) >= std::ldexp(1.0, -126))
            bad++;
        if (std::fabs((double)hi) > std::fabs(x)) bad++;
        if (lo != 0.0f && std::fabs((double)lo) > std::ldexp(std::fabs((double)hi), -23)) bad++;
        if (lo != 0.0f && ((lo < 0) != (x < 0))) bad++;
        if (zolo::df_widen(hi) != (double)hi || zolo::df_widen(lo) != (double)lo) bad++;
    }
    std::printf("worst %.3e bad %d\n", worst, bad);
    return bad == 0 ? 0 : 1;
}
