// Host emulation of the paired-lane 32-point transforms of fft_pair.cuh (no GPU needed): the two
// threads of a pair are run one after the other, with the `send` values swapped by hand where the
// kernel uses a warp shuffle. Checks, with the header's own code:
//  - the DIT and DIF 32-point transforms (both signs) against an FP64 DFT;
//  - the z-pass chain of one 4-column tile of 1024-point lines, stage by stage for every thread
//    (what the block barriers between the stages guarantee), with the exchange-buffer indexing and
//    twiddles of the kernel: the forward transform against an FP64 DFT, and forward then inverse
//    giving back L times the input.
// Exit status 0 when every check passes.
#include <cmath>
#include <cstdio>
#include <vector>

#include "fft_pair.cuh"

using colapm::Tw2;
using colapm::Xch;

static unsigned g_s = 2024u;
static float rnd() {
    g_s = g_s * 1664525u + 1013904223u;
    return (float)((g_s >> 8) * (1.0 / 16777216.0) - 0.5);
}

static void dft_ref(const std::vector<float2>& x, int sign, std::vector<double>& re, std::vector<double>& im) {
    const int n = (int)x.size();
    re.assign(n, 0.0);
    im.assign(n, 0.0);
    for (int k = 0; k < n; ++k)
        for (int m = 0; m < n; ++m) {
            const double a = sign * 2.0 * M_PI * (double)((long long)m * k % n) / n;
            re[k] += x[m].x * std::cos(a) - x[m].y * std::sin(a);
            im[k] += x[m].x * std::sin(a) + x[m].y * std::cos(a);
        }
}

template <int S>
static void pair_dit_host(float2 (*v)[16]) {   // v[h][16]: DFT16 then the exchange, index by index
    for (int h = 0; h < 2; ++h) colapm::dft<16, S>(v[h]);
    for (int i = 0; i < 8; ++i) {
        const float2 s0 = colapm::pair_dit_send(v[0], 0, i), s1 = colapm::pair_dit_send(v[1], 1, i);
        colapm::pair_dit_finish<S>(v[0], 0, i, s1);
        colapm::pair_dit_finish<S>(v[1], 1, i, s0);
    }
}
template <int S>
static void pair_dif_host(float2 (*v)[16]) {
    for (int i = 0; i < 8; ++i) {
        const float2 s0 = colapm::pair_dif_send<S>(v[0], 0, i), s1 = colapm::pair_dif_send<S>(v[1], 1, i);
        colapm::pair_dif_finish(v[0], 0, i, s1);
        colapm::pair_dif_finish(v[1], 1, i, s0);
    }
    for (int h = 0; h < 2; ++h) colapm::pair_dif_dft<S>(v[h]);
}

static double rel(const std::vector<float2>& g, const std::vector<double>& re, const std::vector<double>& im,
                  double scale = 1.0) {
    double e = 0.0, r = 0.0;
    for (size_t k = 0; k < g.size(); ++k) {
        e += std::pow(g[k].x / scale - re[k], 2) + std::pow(g[k].y / scale - im[k], 2);
        r += re[k] * re[k] + im[k] * im[k];
    }
    return std::sqrt(e / r);
}

template <int S>
static int check32() {
    std::vector<float2> x(32), got(32);
    for (auto& e : x) e = make_float2(rnd(), rnd());
    std::vector<double> re, im;
    dft_ref(x, S, re, im);
    // DIT: inputs r = 2m + h in slot m; outputs r = pair_dit_r(q, h) in slot q
    float2 v[2][16];
    for (int h = 0; h < 2; ++h)
        for (int m = 0; m < 16; ++m) v[h][m] = x[2 * m + h];
    pair_dit_host<S>(v);
    for (int h = 0; h < 2; ++h)
        for (int q = 0; q < 16; ++q) got[colapm::pair_dit_r(q, h)] = v[h][q];
    const double e1 = rel(got, re, im);
    // DIF: inputs r = pair_dit_r(q, h) in slot q; outputs 2m + h in slot m
    for (int h = 0; h < 2; ++h)
        for (int q = 0; q < 16; ++q) v[h][q] = x[colapm::pair_dit_r(q, h)];
    pair_dif_host<S>(v);
    for (int h = 0; h < 2; ++h)
        for (int m = 0; m < 16; ++m) got[2 * m + h] = v[h][m];
    const double e2 = rel(got, re, im);
    std::printf("pair DFT32 sign=%+d: DIT rms rel error %.2e, DIF rms rel error %.2e\n", S, e1, e2);
    return e1 < 1e-6 && e2 < 1e-6 ? 0 : 1;
}

static Tw2 tables1024() {
    constexpr int L = 1024;
    Tw2 t;
    auto w = [](long long i) {
        const double a = 2.0 * M_PI * (double)(i % L) / L;
        return make_float2((float)std::cos(a), (float)-std::sin(a));
    };
    for (int j = 0; j < 32; ++j) {
        t.w1[j] = w(j);
        for (int m = 0; m < 4; ++m) t.w8[m][j] = w((long long)8 * m * j);
    }
    return t;
}

// The kernel's chain on one tile of 4 columns (c) x 1024 rows, 256 threads (c, h, j).
static int check_tile() {
    constexpr int L = 1024, R = 32, C = 4;
    using X = Xch<L, R, C>;
    const Tw2 tw = tables1024();
    std::vector<float2> in((size_t)C * L), xb(X::SIZE);
    for (auto& e : in) e = make_float2(rnd(), rnd());
    auto col = [&](int c, int z) -> float2& { return in[(size_t)c * L + z]; };
    float2 reg[C][R][2][16];   // per thread (c, j, h)
    // forward stage A
    for (int c = 0; c < C; ++c)
        for (int j = 0; j < R; ++j) {
            float2 v[2][16];
            for (int h = 0; h < 2; ++h)
                for (int m = 0; m < 16; ++m) v[h][m] = col(c, j + R * (2 * m + h));
            pair_dit_host<-1>(v);
            for (int h = 0; h < 2; ++h)
                for (int q = 0; q < 16; ++q) xb[X::at(c, j * R + colapm::pair_dit_r(q, h))] = v[h][q];
        }
    // forward stage B
    for (int c = 0; c < C; ++c)
        for (int j = 0; j < R; ++j) {
            float2 v[2][16];
            for (int h = 0; h < 2; ++h) {
                for (int m = 0; m < 16; ++m) v[h][m] = xb[X::at(c, j + R * (2 * m + h))];
                colapm::pair_twiddle<-1>(v[h], &tw, j, h);
            }
            pair_dit_host<-1>(v);
            for (int h = 0; h < 2; ++h)
                for (int q = 0; q < 16; ++q) reg[c][j][h][q] = v[h][q];
        }
    int bad = 0;
    double worst = 0.0;
    for (int c = 0; c < C; ++c) {
        std::vector<float2> x(L), got(L);
        for (int z = 0; z < L; ++z) x[z] = col(c, z);
        for (int j = 0; j < R; ++j)
            for (int h = 0; h < 2; ++h)
                for (int q = 0; q < 16; ++q) got[j + R * colapm::pair_dit_r(q, h)] = reg[c][j][h][q];
        std::vector<double> re, im;
        dft_ref(x, -1, re, im);
        worst = std::fmax(worst, rel(got, re, im));
    }
    std::printf("pair z tile forward: rms rel error %.2e\n", worst);
    bad |= worst < 2e-6 ? 0 : 1;
    // inverse stage A (DIF) straight from the forward registers
    for (int c = 0; c < C; ++c)
        for (int j = 0; j < R; ++j) {
            float2 v[2][16];
            for (int h = 0; h < 2; ++h)
                for (int q = 0; q < 16; ++q) v[h][q] = reg[c][j][h][q];
            pair_dif_host<+1>(v);
            for (int h = 0; h < 2; ++h)
                for (int m = 0; m < 16; ++m) xb[X::at(c, j * R + 2 * m + h)] = v[h][m];
        }
    // inverse stage B
    double err = 0.0, ref = 0.0;
    for (int c = 0; c < C; ++c)
        for (int j = 0; j < R; ++j) {
            float2 v[2][16];
            for (int h = 0; h < 2; ++h) {
                for (int m = 0; m < 16; ++m) v[h][m] = xb[X::at(c, j + R * (2 * m + h))];
                colapm::pair_twiddle<+1>(v[h], &tw, j, h);
            }
            pair_dit_host<+1>(v);
            for (int h = 0; h < 2; ++h)
                for (int q = 0; q < 16; ++q) {
                    const float2 a = col(c, j + R * colapm::pair_dit_r(q, h));
                    err += std::pow(v[h][q].x / L - a.x, 2) + std::pow(v[h][q].y / L - a.y, 2);
                    ref += (double)a.x * a.x + (double)a.y * a.y;
                }
        }
    const double rt = std::sqrt(err / ref);
    std::printf("pair z tile forward then inverse: rms rel error %.2e\n", rt);
    bad |= rt < 2e-6 ? 0 : 1;
    return bad;
}

int main() {
    int bad = check32<-1>() | check32<+1>();
    bad |= check_tile();
    return bad;
}
