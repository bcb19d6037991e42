// plan_host.cpp -- FP64 host builders for the plan's coefficient tables:
// windows, windowed-sinc prototypes (Sec. III.A: sinc times a window of length
// N*A_v; Sec. III.B: square-window moving average), NCO word and bin rules.
#include <cmath>
#include <cstdint>

#include "rfr_internal.h"

namespace rfr {

namespace {

constexpr double kPi = 3.14159265358979323846;

// I0(x) = sum_k (x^2/4)^k / (k!)^2, summed to full FP64 precision.
double bessel_i0(double x) {
    const double y = 0.25 * x * x;
    double term = 1.0, acc = 1.0;
    for (int k = 1; k < 2000; ++k) {
        term = term * y / (static_cast<double>(k) * k);
        const double next = acc + term;
        if (next == acc) break;
        acc = next;
    }
    return acc;
}

}  // namespace

// Symmetric window of length m.
int build_window(int kind, double beta, int64_t m, double* w) {
    if (m < 1 || w == nullptr) return -1;
    if (m == 1) {
        w[0] = 1.0;
        return 0;
    }
    const double step = 2.0 * kPi / static_cast<double>(m - 1);
    const double i0b = (kind == RFR_WIN_KAISER) ? bessel_i0(beta) : 1.0;
    for (int64_t j = 0; j < m; ++j) {
        const double c1 = std::cos(step * static_cast<double>(j));
        double v;
        switch (kind) {
        case RFR_WIN_RECT: v = 1.0; break;
        case RFR_WIN_HANN: v = 0.5 * (1.0 - c1); break;
        case RFR_WIN_HAMMING: v = 0.54 - 0.46 * c1; break;
        case RFR_WIN_BLACKMAN: v = 0.42 - 0.5 * c1 + 0.08 * std::cos(2.0 * step * static_cast<double>(j)); break;
        case RFR_WIN_KAISER: {
            const double u = (2.0 * static_cast<double>(j)) / static_cast<double>(m - 1) - 1.0;
            const double arg = 1.0 - u * u;
            v = bessel_i0(beta * std::sqrt(arg > 0.0 ? arg : 0.0)) / i0b;
            break;
        }
        default: return -1;
        }
        w[j] = v;
    }
    return 0;
}

// h[j] = w[j] * sinc(2*fc*(j - (m-1)/2)) (fc <= 0: window only), sum h = 1.
int build_lowpass(int kind, double beta, double fc, int64_t m, double* h) {
    if (build_window(kind, beta, m, h) != 0) return -1;
    if (fc > 0.0) {
        const double mid = 0.5 * static_cast<double>(m - 1);
        for (int64_t j = 0; j < m; ++j) {
            const double u = 2.0 * fc * (static_cast<double>(j) - mid);
            h[j] *= (u == 0.0) ? 1.0 : std::sin(kPi * u) / (kPi * u);
        }
    }
    double sum = 0.0;
    for (int64_t j = 0; j < m; ++j) sum += h[j];
    if (!(std::fabs(sum) > 0.0)) return -1;
    const double inv = 1.0 / sum;
    for (int64_t j = 0; j < m; ++j) h[j] *= inv;
    return 0;
}

uint64_t freq_to_word(double f, double fs) {
    double r = f / fs;
    r = r - std::floor(r + 0.5);                       // [-1/2, 1/2)
    const long long v = std::llround(std::ldexp(r, 64));
    return static_cast<uint64_t>(static_cast<int64_t>(v));
}

int32_t word_to_bin(uint64_t word, int32_t n) {
    // round(word * n / 2^64) mod n, ties up: floor((word*n + 2^63) / 2^64) mod n
    if (n < 2) return -1;
    const unsigned __int128 q = static_cast<unsigned __int128>(word) * static_cast<uint64_t>(n) +
                                (static_cast<unsigned __int128>(1) << 63);
    return static_cast<int32_t>(static_cast<uint64_t>(q >> 64) % static_cast<uint64_t>(n));
}

}  // namespace rfr
