// Host-side check of the bit helpers the key kernels use (bits.cuh).
#include <cstdio>
#include <cstdlib>
#include <set>

#include "../../paper_1610_05108_gb300/csrc/bits.cuh"

int main()
{
    unsigned state = 12345u;
    auto rnd = [&]() { state = state * 1664525u + 1013904223u; return state; };
    for (int trial = 0; trial < 2000; ++trial) {
        uint32_t A[32], B[32];
        for (int i = 0; i < 32; i++) {
            A[i] = rnd();
            if (trial % 3 == 0 && i >= trial % 32)
                A[i] = 0;                          // rows past M are zero
            B[i] = A[i];
        }
        xyz::transpose32(A);
        for (int m = 0; m < 32; m++)
            for (int c = 0; c < 32; c++)
                if (((B[m] >> c) & 1u) != ((A[c] >> m) & 1u)) {
                    std::printf("transpose mismatch trial %d row %d col %d\n", trial, m, c);
                    return 1;
                }
    }
    std::set<uint32_t> seen;
    for (uint32_t x = 0; x < 200000; ++x)
        seen.insert(xyz::mix32(x * 2654435761u));
    if (seen.size() != 200000) {
        std::printf("mix32 collided\n");
        return 1;
    }
    std::printf("ok\n");
    return 0;
}
