// engine.h -- internal declarations shared by the host engine files.
#pragma once
#include <complex>
#include <cstdint>
#include <vector>

namespace fdtd {

struct GridSpec {
    int nx, ny, nz, npml;
    double dx, dy, dz, dt;
};

struct SourceSpec {
    int m;
    double theta;
    int pol;        // 0: Pi_x, 1: Pi_y, 2: circ+, 3: circ-, 4: Pi_z
    int mode;       // 0: TE, 1: TM
    double E0;
    double r_center, thickness;
    int inject;     // 0: all components, 1: tangential
};

double bessel_j(int n, double x);
void beam_fields(const SourceSpec& s, double x, double y, double z,
                 std::complex<double> E[3], std::complex<double> H[3]);
int component_z_half(int c);
bool ring_contains(const GridSpec& g, const SourceSpec& s, int c, int i, int j);
void source_tables(const GridSpec& g, const SourceSpec& s, const double* w_amp,
                   const double* w_phase, std::vector<std::complex<double>>& coef,
                   std::vector<uint8_t>& mask, int64_t counts[6]);

}  // namespace fdtd
