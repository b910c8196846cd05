// source_precompute.cpp -- host FP64 precompute of the Bessel-antenna source.
//
// For every transverse column (i, j) and field component c this computes the
// complex amplitude A_c(x, y, z0) of the order-m vector Bessel beam at the
// component's Yee position (z0 = 0 for Ex, Ey, Hz; dz/2 for Ez, Hx, Hy) and
// the antenna mask (which columns hold a point of the hollow annulus, Fig. 3).
// The kernels multiply A by e^{i beta k dz} (a per-plane table) and by
// e^{-i omega t'} f(t) (per step), Eq. 12-13.
//
// Formulation.  The Hertz potential of Eq. 5 is Pi = p psi with
// psi = J_m(K r) e^{i m phi} e^{i beta z} (K = k sin theta, beta = k cos theta,
// read with e^{+i beta z} e^{-i omega t}: the convention the printed Q and R of
// Eq. 6-7 follow).  With g = grad psi and G = grad grad psi:
//     Q = curl(p psi) = g x p,    R = curl curl(p psi) = G p + k^2 p psi,
// which reproduces Eq. 6 (p = x), Eq. 7 (p = y) and their complex
// combinations (circular polarisation).  The derivatives use the ladder
// relations (d_x +- i d_y)[J_n(Kr) e^{i n phi}] = -+ K J_{n+-1}(Kr) e^{i(n+-1)phi}.
// TE (Eq. 9a): E = (E0/k) Q, H = -i (E0/k^2) R.  TM (Eq. 9b): E = (E0/k^2) R,
// H = -i (E0/k) Q.  The -i on H is Faraday's law for e^{-i omega t}
// (H = curl E / (i omega mu0)); Eq. 12b prints the magnetic term without it.
//
// Bessel functions: Miller's backward recurrence (J. C. P. Miller, 1952;
// Abramowitz & Stegun 9.12; the normalisation 1 = J_0 + 2 sum_k J_2k is
// Abramowitz & Stegun 9.1.46), J_{-n} = (-1)^n J_n.
#include <cmath>
#include <complex>
#include <cstdint>
#include <vector>

#include "engine.h"

namespace fdtd {

using cd = std::complex<double>;

double bessel_j(int n, double x)
{
    if (n < 0) {
        double v = bessel_j(-n, x);
        return ((-n) & 1) ? -v : v;
    }
    if (x < 0.0) {
        double v = bessel_j(n, -x);
        return (n & 1) ? -v : v;
    }
    if (x == 0.0) return n == 0 ? 1.0 : 0.0;
    // Start the downward recurrence far above both n and x; an even start
    // order keeps the normalisation sum aligned with the even orders.
    int start = n + static_cast<int>(x) + 40 + static_cast<int>(std::sqrt(40.0 * (n + x + 1.0)));
    start += start & 1;
    double jp = 0.0;       // J_{k+1} (unnormalised)
    double jk = 1e-300;    // J_k
    double norm = 0.0;     // J_0 + 2 sum J_{2k}
    double result = 0.0;
    for (int k = start; k > 0; --k) {
        double jm = (2.0 * k / x) * jk - jp;   // J_{k-1}
        jp = jk;
        jk = jm;
        if (std::fabs(jk) > 1e250) {           // rescale to stay in range
            jk *= 1e-250; jp *= 1e-250; norm *= 1e-250; result *= 1e-250;
        }
        int order = k - 1;
        if (order == n) result = jk;
        if (order > 0 && (order & 1) == 0) norm += 2.0 * jk;
    }
    norm += jk;   // J_0
    if (n == 0) result = jk;
    return result / norm;
}

namespace {

struct Derivs {
    cd psi;          // psi at (x, y, 0)
    cd g[3];         // gradient
    cd G[3][3];      // Hessian
};

// psi and its first and second derivatives at (x, y, z = 0) for order m.
Derivs potential_derivs(int m, double K, double beta, double x, double y)
{
    double r = std::sqrt(x * x + y * y);
    double phi = r > 0.0 ? std::atan2(y, x) : 0.0;
    // L_n = J_n(K r) e^{i n phi} for the orders the ladder reaches
    auto L = [&](int n) { return bessel_j(n, K * r) * std::polar(1.0, n * phi); };
    cd l0 = L(m), lp1 = L(m + 1), lm1 = L(m - 1), lp2 = L(m + 2), lm2 = L(m - 2);
    const cd I(0.0, 1.0);
    // d+ = dx + i dy, d- = dx - i dy:  d+ L_n = -K L_{n+1},  d- L_n = K L_{n-1}
    cd dp = -K * lp1, dm = K * lm1;
    cd dpp = K * K * lp2, dmm = K * K * lm2, dpm = -K * K * l0;
    Derivs d;
    d.psi = l0;
    d.g[0] = 0.5 * (dp + dm);
    d.g[1] = (dp - dm) / (2.0 * I);
    d.g[2] = I * beta * l0;
    cd dxx = 0.25 * (dpp + 2.0 * dpm + dmm);
    cd dyy = -0.25 * (dpp - 2.0 * dpm + dmm);
    cd dxy = (dpp - dmm) / (4.0 * I);
    cd dxz = I * beta * d.g[0], dyz = I * beta * d.g[1], dzz = -beta * beta * l0;
    d.G[0][0] = dxx; d.G[0][1] = dxy; d.G[0][2] = dxz;
    d.G[1][0] = dxy; d.G[1][1] = dyy; d.G[1][2] = dyz;
    d.G[2][0] = dxz; d.G[2][1] = dyz; d.G[2][2] = dzz;
    return d;
}

}  // namespace

void beam_fields(const SourceSpec& s, double x, double y, double z, cd E[3], cd H[3])
{
    const double k = 2.0 * M_PI;
    double K = k * std::sin(s.theta), beta = k * std::cos(s.theta);
    const cd I(0.0, 1.0);
    cd p[3];
    switch (s.pol) {
        case 0: p[0] = 1.0; p[1] = 0.0; p[2] = 0.0; break;              // Pi_x
        case 1: p[0] = 0.0; p[1] = 1.0; p[2] = 0.0; break;              // Pi_y
        case 2: p[0] = 1.0 / std::sqrt(2.0); p[1] = I / std::sqrt(2.0); p[2] = 0.0; break;
        case 4: p[0] = 0.0; p[1] = 0.0; p[2] = 1.0; break;              // Pi_z
        default: p[0] = 1.0 / std::sqrt(2.0); p[1] = -I / std::sqrt(2.0); p[2] = 0.0; break;
    }
    Derivs d = potential_derivs(s.m, K, beta, x, y);
    cd zf = std::polar(1.0, beta * z);
    cd Q[3], R[3];
    // Q = g x p
    Q[0] = d.g[1] * p[2] - d.g[2] * p[1];
    Q[1] = d.g[2] * p[0] - d.g[0] * p[2];
    Q[2] = d.g[0] * p[1] - d.g[1] * p[0];
    for (int a = 0; a < 3; ++a) {
        R[a] = k * k * p[a] * d.psi;
        for (int b = 0; b < 3; ++b) R[a] += d.G[a][b] * p[b];
    }
    for (int a = 0; a < 3; ++a) {
        if (s.mode == 0) {
            E[a] = (s.E0 / k) * Q[a] * zf;
            H[a] = -I * (s.E0 / (k * k)) * R[a] * zf;
        } else {
            E[a] = (s.E0 / (k * k)) * R[a] * zf;
            H[a] = -I * (s.E0 / k) * Q[a] * zf;
        }
    }
    if (s.inject == 1) {
        double r = std::sqrt(x * x + y * y);
        if (r > 0.0) {
            double ux = x / r, uy = y / r;
            cd er = E[0] * ux + E[1] * uy, hr = H[0] * ux + H[1] * uy;
            E[0] -= er * ux; E[1] -= er * uy;
            H[0] -= hr * ux; H[1] -= hr * uy;
        }
    }
}

// Staggered offsets (cells) of Ex, Ey, Ez, Hx, Hy, Hz (x, y, z).
static const double kOff[6][3] = {
    {0.5, 0.0, 0.0}, {0.0, 0.5, 0.0}, {0.0, 0.0, 0.5},
    {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}, {0.5, 0.5, 0.0},
};

int component_z_half(int c) { return kOff[c][2] != 0.0 ? 1 : 0; }

bool ring_contains(const GridSpec& g, const SourceSpec& s, int c, int i, int j)
{
    // The membership decision is made on exact half-integer cell offsets.
    double rin = s.r_center - 0.5 * s.thickness;
    double rout = s.r_center + 0.5 * s.thickness;
    double u = i + kOff[c][0] - 0.5 * g.nx, v = j + kOff[c][1] - 0.5 * g.ny;
    double r2 = u * u + v * v;
    if (!(r2 >= rin * rin && r2 < rout * rout)) return false;
    if ((c == 1 || c == 2) && i == 0) return false;   // PEC-clamped tangential E
    if ((c == 0 || c == 2) && j == 0) return false;
    return true;
}

void source_tables(const GridSpec& g, const SourceSpec& s, const double* w_amp,
                   const double* w_phase, std::vector<cd>& coef, std::vector<uint8_t>& mask,
                   int64_t counts[6])
{
    const size_t ncol = static_cast<size_t>(g.nx) * g.ny;
    coef.assign(6 * ncol, cd(0.0, 0.0));
    mask.assign(ncol, 0);
    for (int c = 0; c < 6; ++c) counts[c] = 0;
    for (int j = 0; j < g.ny; ++j)
        for (int i = 0; i < g.nx; ++i) {
            size_t col = static_cast<size_t>(j) * g.nx + i;
            for (int c = 0; c < 6; ++c) {
                if (!ring_contains(g, s, c, i, j)) continue;
                double x = (i + kOff[c][0] - 0.5 * g.nx) * g.dx;
                double y = (j + kOff[c][1] - 0.5 * g.ny) * g.dy;
                double z = kOff[c][2] * g.dz;
                cd E[3], H[3];
                beam_fields(s, x, y, z, E, H);
                cd a = c < 3 ? E[c] : H[c - 3];
                double wa = w_amp ? w_amp[col] : 1.0;
                double wp = w_phase ? w_phase[col] : 0.0;
                coef[c * ncol + col] = std::polar(wa, wp) * a;
                mask[col] |= static_cast<uint8_t>(1u << c);
                counts[c] += g.nz;
            }
        }
}

}  // namespace fdtd
