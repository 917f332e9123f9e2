// CPU check of the integer FP32-pair split (pairsplit.h) against its FP64 definition
// hi = (float)v, lo = (float)(v - (double)hi), bit for bit, and of the exact widening.
#include <math.h>
#include <stdio.h>
#include <stdint.h>
#include <string.h>

#include <limits>
#include <random>

#include "pairsplit.h"

static uint32_t fb(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static uint64_t db(double d) { uint64_t u; memcpy(&u, &d, 8); return u; }

static int check(double v) {
    float hi, lo;
    helm::split_double_int(v, hi, lo);
    const float rh = (float)v;
    const float rl = (float)(v - (double)rh);
    const bool nan_ok = isnan(rh) && isnan(hi);
    if (!nan_ok && (fb(hi) != fb(rh) || fb(lo) != fb(rl))) {
        printf("mismatch v=%.17g (bits %016llx): hi %a vs %a, lo %a vs %a\n", v, (unsigned long long)db(v), hi, rh, lo,
               rl);
        return 1;
    }
    // widening: exactly (double)hi + (double)lo
    if (!isnan(v)) {
        const double w = helm::pair_to_double(hi, lo), ref = (double)hi + (double)lo;
        if (db(w) != db(ref)) {
            printf("widening v=%.17g: %.17g vs %.17g\n", v, w, ref);
            return 1;
        }
    }
    return 0;
}

int main() {
    int bad = 0;
    const double specials[] = {0.0, -0.0, 1.0, -1.0, 1.5, 3.0, 1e-300, -1e-300, 4.9e-324, 1e300, -1e300,
                               std::numeric_limits<double>::infinity(), -std::numeric_limits<double>::infinity(),
                               std::numeric_limits<double>::quiet_NaN(), 3.4028234663852886e38, 3.4028235677973366e38,
                               1.1754943508222875e-38, 5.877471754111438e-39, 0x1.fffffffp0, 0x1.ffffffp+126,
                               0x1.0000001p0, 0x1.0000003p0, 0x1.00000030000001p0, -0x1.0000001p-74, 0x1p-74, 0x1p-75,
                               0x1p126, 0x1.fffffffffffffp126, 0x1p127};
    for (double v : specials) bad += check(v);
    std::mt19937_64 rng(12345);
    for (int i = 0; i < 2000000 && bad < 10; ++i) {
        uint64_t u = rng();
        if (i % 4 == 0) {   // exponents around the float range's edges and the branch limits
            const int e = 1023 + (int)(rng() % 260) - 130;
            u = (u & 0x800FFFFFFFFFFFFFull) | ((uint64_t)e << 52);
        } else if (i % 4 == 1) {   // significands at and next to the rounding ties
            const int e = 1023 + (int)(rng() % 200) - 100;
            const uint64_t tie = (1ull << 28) + (uint64_t)((int)(rng() % 5) - 2);
            u = (u & 0x800FFFFFE0000000ull) | ((uint64_t)e << 52) | tie;
            u = (u & ~(0x7FFull << 52)) | ((uint64_t)e << 52);
        }
        double v;
        memcpy(&v, &u, 8);
        bad += check(v);
    }
    if (bad) return 1;
    printf("ok\n");
    return 0;
}
