// Host-side check of the half-spectrum index maps of the two-stage FFT passes (no GPU needed):
// hs_index<L, BLK> must map (kx < L/2, y < L, z < L) one-to-one onto [0, L/2 L L), and hs_ystep(d)
// must be the distance between rows y and y + d of one column whenever d is a multiple of 8 (the
// register strides of the y passes). Exit status 0 when every check passes.
#include <cstdio>
#include <vector>

#include "fft2.cuh"

template <int L, bool BLK>
static int check() {
    const size_t n = (size_t)(L / 2) * L * L;
    std::vector<unsigned char> seen(n, 0);
    for (int z = 0; z < L; ++z)
        for (int y = 0; y < L; ++y)
            for (int kx = 0; kx < L / 2; ++kx) {
                const size_t i = colapm::hs_index<L, BLK>(kx, y, z);
                if (i >= n || seen[i]) {
                    std::printf("L=%d BLK=%d: index %zu of (%d,%d,%d) %s\n", L, (int)BLK, i, kx, y, z,
                                i >= n ? "out of range" : "repeated");
                    return 1;
                }
                seen[i] = 1;
            }
    for (int d = 8; d < L; d *= 2)
        for (int y = 0; y + d < L; y += 3)
            for (int kx = 0; kx < L / 2; kx += 7)
                for (int z = 0; z < L; z += 97) {
                    const size_t a = colapm::hs_index<L, BLK>(kx, y, z), b = colapm::hs_index<L, BLK>(kx, y + d, z);
                    if (b - a != colapm::hs_ystep<L, BLK>(d)) {
                        std::printf("L=%d BLK=%d: row step %d at (%d,%d,%d) is %zu, not %zu\n", L, (int)BLK, d, kx, y,
                                    z, b - a, colapm::hs_ystep<L, BLK>(d));
                        return 1;
                    }
                }
    std::printf("L=%d BLK=%d: %zu indices one-to-one, row steps consistent\n", L, (int)BLK, n);
    return 0;
}

int main() {
    int bad = 0;
    bad |= check<256, false>();
    bad |= check<512, false>();
    bad |= check<512, true>();
    bad |= check<1024, true>();
    return bad;
}
