// Host-side check of the construction behind the class-split survivor
// filter: the class of an M-bit key (bit b = parity of the key bits m with
// m % 4 == b) is linear over GF(2), and planes formed as the XOR of the
// sampled row words m = b (mod 4), placed in rows 28-31 of the 32 x 32
// transpose, come out as each column's class in the top four bits.
#include <cstdio>

#include "../../paper_1610_05108_gb300/csrc/bits.cuh"

static uint32_t parity(uint32_t x)
{
    uint32_t p = 0;
    while (x) {
        p ^= 1u;
        x &= x - 1;
    }
    return p;
}

// the definition, one key bit at a time
static uint32_t key_class_def(uint32_t k, int M)
{
    uint32_t q = 0;
    for (int m = 0; m < M; ++m)
        if ((k >> m) & 1u)
            q ^= 1u << (m & 3);
    return q;
}

int main()
{
    unsigned state = 777u;
    auto rnd = [&]() { state = state * 1664525u + 1013904223u; return state; };
    for (int M = 1; M <= 28; ++M) {
        const uint32_t kmask = (M == 32) ? ~0u : ((1u << M) - 1u);
        // linearity: class(k ^ c) = class(k) ^ class(c); and the masked-parity
        // form used on the device agrees with the definition
        for (int trial = 0; trial < 2000; ++trial) {
            const uint32_t k = rnd() & kmask, c = rnd() & kmask;
            if (key_class_def(k ^ c, M) != (key_class_def(k, M) ^ key_class_def(c, M))) {
                std::printf("class not linear, M %d\n", M);
                return 1;
            }
            uint32_t q = 0;
            for (int b = 0; b < 4; ++b)
                q |= parity(k & (0x11111111u << b)) << b;
            if (q != key_class_def(k, M)) {
                std::printf("masked parity differs, M %d\n", M);
                return 1;
            }
            // round matching: k ^ c has class q exactly when k has class q ^ class(c)
            for (uint32_t qq = 0; qq < 16; ++qq)
                if ((key_class_def(k ^ c, M) == qq) != (key_class_def(k, M) == (qq ^ key_class_def(c, M)))) {
                    std::printf("round matching fails, M %d\n", M);
                    return 1;
                }
        }
        // the class planes carried through the transpose
        for (int trial = 0; trial < 300; ++trial) {
            uint32_t A[32] = {0};
            for (int m = 0; m < M; ++m)
                A[m] = rnd();
            uint32_t Q[4] = {0, 0, 0, 0};
            for (int m = 0; m < M; ++m)
                Q[m & 3] ^= A[m];
            for (int b = 0; b < 4; ++b)
                A[28 + b] = Q[b];
            uint32_t rows[32];
            for (int m = 0; m < 32; ++m)
                rows[m] = A[m];
            xyz::transpose32(A);
            for (int cc = 0; cc < 32; ++cc) {
                uint32_t key = 0;
                for (int m = 0; m < M; ++m)
                    key |= ((rows[m] >> cc) & 1u) << m;
                if ((A[cc] & kmask) != key || (A[cc] >> 28) != key_class_def(key, M)) {
                    std::printf("transposed class differs, M %d column %d\n", M, cc);
                    return 1;
                }
            }
        }
    }
    std::printf("ok\n");
    return 0;
}
