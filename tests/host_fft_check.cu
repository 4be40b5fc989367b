// Host emulation of the two-stage register FFT of fft2.cuh (no GPU needed). The passes separate
// their two stages with a block barrier, so running stage A for every task, then stage B for every
// task, reproduces a tile exactly. The checks use the header's own DFT, twiddle and exchange-buffer
// code:
//  - every composite register radix (prime-factor split) against an FP64 DFT;
//  - forward (radices R1, R2) and inverse transforms of 8 lines against an FP64 DFT, at every
//    length with a two-stage plan (64 ... 1024, including the mixed 96, 160, 192, 320, 384);
//  - the z-pass chain: the forward stage-B outputs of task j, fed unchanged to stage A of the
//    inverse with the radices swapped, give back L times the input.
// Exit status 0 when every check passes.
#include <cmath>
#include <cstdio>
#include <vector>

#include "fft2.cuh"

using colapm::Tw2;
using colapm::Xch;

template <int L>
static Tw2 tables() {   // w1[j] = w^j, w8[m][j] = w^(8 m j), w = exp(-2 pi i / L), as the library fills them
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

// one two-stage transform of 8 lines (sign S), radices RA then RB; out[c][k] in natural order
template <int L, int RA, int RB, int S>
static void transform(const std::vector<float2>& in, std::vector<float2>& out, const Tw2& tw) {
    std::vector<float2> xb(Xch<L, RA>::SIZE);
    for (int c = 0; c < 8; ++c)
        for (int j = 0; j < L / RA; ++j) {   // stage A
            float2 v[RA];
            for (int r = 0; r < RA; ++r) v[r] = in[c * L + j + r * (L / RA)];
            colapm::dft<RA, S>(v);
            for (int r = 0; r < RA; ++r) xb[Xch<L, RA>::at(c, j * RA + r)] = v[r];
        }
    for (int c = 0; c < 8; ++c)
        for (int j = 0; j < RA; ++j) {       // stage B
            float2 v[RB];
            colapm::stage_b<L, RA, RB, S>(xb.data(), &tw, c, j, v);
            for (int r = 0; r < RB; ++r) out[c * L + j + RA * r] = v[r];
        }
}

template <int L>
static int check() {
    constexpr int R1 = colapm::F2<L>::R1, R2 = colapm::F2<L>::R2;
    const Tw2 tw = tables<L>();
    std::vector<float2> x(8 * L), X(8 * L), y(8 * L);
    unsigned s = 12345u + L;
    auto rnd = [&s] { s = s * 1664525u + 1013904223u; return (float)((s >> 8) * (1.0 / 16777216.0) - 0.5); };
    for (auto& e : x) e = make_float2(rnd(), rnd());
    for (int dir = -1; dir <= 1; dir += 2) {
        if (dir < 0) transform<L, R1, R2, -1>(x, X, tw);
        else transform<L, R1, R2, +1>(x, X, tw);
        double err = 0.0, ref = 0.0;
        for (int c = 0; c < 8; ++c)
            for (int k = 0; k < L; ++k) {   // FP64 DFT
                double re = 0.0, im = 0.0;
                for (int m = 0; m < L; ++m) {
                    const double a = dir * 2.0 * M_PI * (double)((long long)m * k % L) / L;
                    const float2 v = x[c * L + m];
                    re += v.x * std::cos(a) - v.y * std::sin(a);
                    im += v.x * std::sin(a) + v.y * std::cos(a);
                }
                const float2 g = X[c * L + k];
                err += (g.x - re) * (g.x - re) + (g.y - im) * (g.y - im);
                ref += re * re + im * im;
            }
        const double rel = std::sqrt(err / ref);
        std::printf("L=%d sign=%+d: rms rel error %.2e\n", L, dir, rel);
        if (!(rel < 2e-6)) return 1;
    }
    // z-pass chain: forward (R1, R2); the outputs X[j + R1 r] of task j are the inputs of task j of
    // the inverse with radices (R2, R1)
    transform<L, R1, R2, -1>(x, X, tw);
    std::vector<float2> xb(Xch<L, R2>::SIZE);
    for (int c = 0; c < 8; ++c)
        for (int j = 0; j < R1; ++j) {
            float2 v[R2];
            for (int r = 0; r < R2; ++r) v[r] = X[c * L + j + R1 * r];
            colapm::dft<R2, +1>(v);
            for (int r = 0; r < R2; ++r) xb[Xch<L, R2>::at(c, j * R2 + r)] = v[r];
        }
    double err = 0.0, ref = 0.0;
    for (int c = 0; c < 8; ++c)
        for (int j = 0; j < R2; ++j) {
            float2 u[R1];
            colapm::stage_b<L, R2, R1, +1>(xb.data(), &tw, c, j, u);
            for (int r = 0; r < R1; ++r) {
                const float2 a = x[c * L + j + R2 * r];
                err += std::pow(u[r].x / L - a.x, 2) + std::pow(u[r].y / L - a.y, 2);
                ref += (double)a.x * a.x + (double)a.y * a.y;
            }
        }
    const double rel = std::sqrt(err / ref);
    std::printf("L=%d forward then swapped-radix inverse: rms rel error %.2e\n", L, rel);
    return rel < 2e-6 ? 0 : 1;
}

// One R-point register DFT (composite R: the prime-factor split) against an FP64 DFT, both signs.
template <int R>
static int check_radix() {
    unsigned s = 777u + R;
    auto rnd = [&s] { s = s * 1664525u + 1013904223u; return (float)((s >> 8) * (1.0 / 16777216.0) - 0.5); };
    float2 x[R];
    for (auto& e : x) e = make_float2(rnd(), rnd());
    double worst = 0.0;
    for (int dir = -1; dir <= 1; dir += 2) {
        float2 v[R];
        for (int m = 0; m < R; ++m) v[m] = x[m];
        if (dir < 0) colapm::dft<R, -1>(v);
        else colapm::dft<R, +1>(v);
        double err = 0.0, ref = 0.0;
        for (int k = 0; k < R; ++k) {
            double re = 0.0, im = 0.0;
            for (int m = 0; m < R; ++m) {
                const double a = dir * 2.0 * M_PI * (double)(m * k % R) / R;
                re += x[m].x * std::cos(a) - x[m].y * std::sin(a);
                im += x[m].x * std::sin(a) + x[m].y * std::cos(a);
            }
            err += (v[k].x - re) * (v[k].x - re) + (v[k].y - im) * (v[k].y - im);
            ref += re * re + im * im;
        }
        worst = std::fmax(worst, std::sqrt(err / ref));
    }
    std::printf("radix %d: rms rel error %.2e\n", R, worst);
    return worst < 1e-6 ? 0 : 1;
}

int main() {
    int bad = 0;
    bad |= check_radix<6>() | check_radix<10>() | check_radix<12>() | check_radix<15>() | check_radix<20>() |
           check_radix<24>() | check_radix<40>() | check_radix<48>();
    bad |= check<64>();
    bad |= check<96>();
    bad |= check<128>();
    bad |= check<160>();
    bad |= check<192>();
    bad |= check<256>();
    bad |= check<320>();
    bad |= check<384>();
    bad |= check<512>();
    bad |= check<1024>();
    return bad;
}
