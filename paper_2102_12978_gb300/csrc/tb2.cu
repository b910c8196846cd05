// tb2.cu -- launch of the two-step temporally blocked kernel yee_tb2 (tile
// variant 7): windows, the flattened (window, plane) work split into ranges
// of equal estimated cost over one wave of resident CTAs, and the source time
// factors of both steps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "grid_impl.h"
#include "yee_tb2.cuh"

namespace fdtd {

void tb2_windows(const fdtd_grid_desc& d, int ry, int* t, int* u)
{
    *t = d.nx <= kTb2Wx ? 1 : (d.nx - kTb2Wx + kTb2Sx - 1) / kTb2Sx + 1;
    *u = d.ny <= ry ? 1 : (d.ny - ry + (ry - 4) - 1) / (ry - 4) + 1;
}

std::vector<long long> tb2_refined_ranges(const std::vector<long long>& s, const unsigned long long* cycles,
                                          double step)
{
    const int slots = int(s.size()) - 1;
    double total = 0.0;
    for (int c = 0; c < slots; ++c)
        if (s[size_t(c) + 1] > s[size_t(c)]) total += double(cycles[c]);
    if (!(total > 0.0)) return s;
    // cost of the items [0, x): piecewise linear, CTA c's items at cycles_c / (its item count) each
    std::vector<long long> ns(size_t(slots) + 1, s.back());
    ns[0] = 0;
    int c = 0;
    double cum = 0.0;
    for (int k = 1; k < slots; ++k) {
        const double target = total * k / slots;
        while (c < slots && (s[size_t(c) + 1] == s[size_t(c)] || cum + double(cycles[c]) < target)) {
            if (s[size_t(c) + 1] > s[size_t(c)]) cum += double(cycles[c]);
            ++c;
        }
        double x = double(s.back());
        if (c < slots) {
            const double frac = (target - cum) / double(cycles[c]);
            x = double(s[size_t(c)]) + frac * double(s[size_t(c) + 1] - s[size_t(c)]);
        }
        // move the boundary `step` of the way (damping against oscillation)
        const long long y = std::llround(double(s[size_t(k)]) + step * (x - double(s[size_t(k)])));
        ns[size_t(k)] = std::max(ns[size_t(k) - 1], std::min(y, s.back()));
    }
    return ns;
}

void tb2_refine(fdtd_grid* g, int ry, int slots, const unsigned long long* cycles, double step)
{
    // the ranges the measured launches ran: the cached plan of this shape
    if (g->tb2_key.ry != ry || g->tb2_key.slots != slots || g->tb2_start.size() != size_t(slots) + 1) return;
    g->tb2_refined = tb2_refined_ranges(g->tb2_start, cycles, step);
    g->tb2_ref_order = g->tb2_key.order;
    g->tb2_ref_ry = ry;
    g->tb2_ref_slots = slots;
    g->tb2_ref_src = g->src_gen;
    g->tb2_ref_gen += 1;
}

// Rows interleaved by D (see Tb2Plan) for window order `mode` 2, row by row
// (D = 1) otherwise: D in [1, 16] such that D windows of planes come closest
// to a whole number of CTA shares.
static int tb2_order_d(int T, int U, int nz, int slots, int mode)
{
    if (mode != 2) return 1;
    const double share = double(T) * U * nz / slots;
    int best = 1;
    double bd = 1e30;
    for (int D = 1; D <= 16 && D <= U; ++D) {
        const double r = std::fmod(double(nz) * D, share), dist = std::min(r, share - r);
        if (dist < bd - 1e-9) { bd = dist; best = D; }
    }
    return best;
}

// Window at flattened position pos (the host copy of tb2_window_at).
static int tb2_window_host(int T, int U, int D, int pos)
{
    if (D <= 1) return pos;
    const int grp = pos / (T * D);
    const int rows = std::min(D, U - grp * D);
    const int r = pos - grp * T * D;
    const int wx = r / rows, l = r - wx * rows;
    return (grp * D + l) * T + wx;
}

// CTA work ranges of variant 7 on grid g: windows of 32 x RY columns, `slots`
// resident CTAs.  Each CTA gets a contiguous range of (window, plane) items.
// The ranges either have equal estimated cost -- a window-plane costs 1,
// plus w_shell if the window holds CPML shell columns, plus w_ant if it holds
// antenna columns, and a window costs kRestart more planes at its start (the
// wavefront refills) -- or (tc.measured) are the ones tb2_refine moved until
// the CTAs' measured times were equal.  Cached on the grid until the antenna,
// the weights or the launch shape change.
constexpr double kRestart = 3.0;
static void tb2_plan(fdtd_grid* g, int RY, int slots, const TileConfig& tc, Tb2Plan& P)
{
    const fdtd_grid_desc& d = g->desc;
    tb2_windows(d, RY, &P.T, &P.U);
    P.prof = nullptr;
    const int order = tc.lz == 2 ? 2 : 1;
    P.D = tb2_order_d(P.T, P.U, d.nz, slots, order);
    const bool meas = tc.measured && g->tb2_ref_ry == RY && g->tb2_ref_slots == slots &&
                      g->tb2_ref_src == g->src_gen && g->tb2_refined.size() == size_t(slots) + 1 &&
                      g->tb2_ref_order == order;
    auto& key = g->tb2_key;
    if (key.ry != RY || key.slots != slots || key.src_gen != g->src_gen || key.measured != meas ||
        key.order != order ||
        (meas ? key.cost_gen != g->tb2_ref_gen : (key.w_shell != tc.w_shell || key.w_ant != tc.w_ant))) {
        if (meas) {
            g->tb2_start = g->tb2_refined;
        } else {
            const int nx = d.nx, ny = d.ny, nz = d.nz, npml = d.npml;
            const int nw = P.T * P.U;
            std::vector<double> cost(size_t(nw), 1.0);
            for (int wy = 0; wy < P.U; ++wy)
                for (int wx = 0; wx < P.T; ++wx) {
                    const int i0 = kTb2Sx * wx, i1 = std::min(i0 + kTb2Wx, nx);
                    const int j0 = (RY - 4) * wy, j1 = std::min(j0 + RY, ny);
                    const bool shell = npml > 0 && (i0 < npml || i1 > nx - npml || j0 < npml || j1 > ny - npml);
                    bool ant = false;
                    if (!g->hmask.empty())
                        for (int j = j0; j < j1 && !ant; ++j)
                            for (int i = i0; i < i1 && !ant; ++i) ant = g->hmask[size_t(j) * nx + i] != 0;
                    cost[size_t(wy) * P.T + wx] = 1.0 + (shell ? tc.w_shell : 0.0) + (ant ? tc.w_ant : 0.0);
                }
            if (P.D > 1) {   // costs by position
                std::vector<double> byp(cost.size());
                for (int m = 0; m < nw; ++m) byp[size_t(m)] = cost[size_t(tb2_window_host(P.T, P.U, P.D, m))];
                cost.swap(byp);
            }
            double total = 0.0;
            for (double c : cost) total += c * (nz + kRestart);
            const double share = total / slots;
            std::vector<long long> start(size_t(slots) + 1, (long long)nw * nz);
            start[0] = 0;
            int c = 1;
            double cum = 0.0;
            for (int w = 0; w < nw && c < slots; ++w) {
                const double cw = cost[size_t(w)];
                const double span = cw * (nz + kRestart), base = cum + cw * kRestart;
                while (c < slots && c * share < cum + span) {
                    long long k = (long long)std::ceil((c * share - base) / cw);
                    k = std::max(0LL, std::min((long long)nz, k));
                    start[size_t(c)] = std::max(start[size_t(c) - 1], (long long)w * nz + k);
                    ++c;
                }
                cum += span;
            }
            g->tb2_start = start;
        }
        key.ry = RY; key.slots = slots; key.src_gen = g->src_gen;
        key.w_shell = tc.w_shell; key.w_ant = tc.w_ant;
        key.measured = meas; key.cost_gen = g->tb2_ref_gen; key.order = order;
    }
    for (int c = 0; c <= slots; ++c) P.start[c] = g->tb2_start[size_t(c)];
}

// Resident CTAs per SM of the kernels of one RY (dynamic shared memory set
// on first use).
template <int RY>
static cudaError_t tb2_blocks_per_sm(int* out)
{
    using S = Tb2Smem<RY>;
    static_assert(S::bytes() <= 232448, "the window's shared memory exceeds the 227 KB a CTA can hold");
    static int blocks_per_sm = 0;
    if (blocks_per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(yee_tb2<RY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(S::bytes()));

        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(yee_tb2_t<RY>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(S::bytes()));
        if (e != cudaSuccess) return e;
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, yee_tb2<RY>, 32 * RY, S::bytes());
        if (e != cudaSuccess) return e;
        if (n < 1) return cudaErrorInvalidConfiguration;
        blocks_per_sm = n;
    }
    *out = blocks_per_sm;
    return cudaSuccess;
}

int tb2_slots(const fdtd_grid* g, int ry)
{
    int per_sm = 0;
    const cudaError_t e = ry == 8 ? tb2_blocks_per_sm<8>(&per_sm) : tb2_blocks_per_sm<16>(&per_sm);
    if (e != cudaSuccess) return -1;
    return std::min(kTb2MaxCtas, (g->sm_count > 0 ? g->sm_count : 152) * per_sm);
}

template <int RY>
static cudaError_t launch_tb2_t(const fdtd_grid* cg, int cur, long long n, const TileConfig& tc, cudaStream_t s)
{
    fdtd_grid* g = const_cast<fdtd_grid*>(cg);
    using S = Tb2Smem<RY>;
    int per_sm = 0;
    cudaError_t e = tb2_blocks_per_sm<RY>(&per_sm);
    if (e != cudaSuccess) return e;
    const int slots = std::min(kTb2MaxCtas, (g->sm_count > 0 ? g->sm_count : 152) * per_sm);
    Tb2Plan plan;
    tb2_plan(g, RY, slots, tc, plan);
    if (g->tb2_profile)
        plan.prof = reinterpret_cast<unsigned long long*>(static_cast<char*>(g->arena) + g->L.tb2prof);
    const StepTime<float> t0 = step_time<float>(g->srct, nullptr, g->dt, n);
    const StepTime<float> t1 = step_time<float>(g->srct, nullptr, g->dt, n + 1);
    Tb2Times tt;
    tt.th0 = t0.th; tt.te0 = t0.te; tt.th1 = t1.th; tt.te1 = t1.te;
    yee_tb2<RY><<<unsigned(slots), dim3(32, RY), S::bytes(), s>>>(make_args<float>(g, cur), tt, plan);
    return cudaGetLastError();
}

cudaError_t launch_tb2(const fdtd_grid* g, int cur, long long n, const TileConfig& tc, cudaStream_t s)
{
    if (g->desc.precision != FDTD_F32 || needs_cell_passes(g)) return cudaErrorInvalidValue;
    if (tc.ty == 8) return launch_tb2_t<8>(g, cur, n, tc, s);
    return launch_tb2_t<16>(g, cur, n, tc, s);
}

cudaError_t launch_tb2_table(const fdtd_grid* cg, int cur, const StepTime<float>* times, int i0, int i1,
                             int max_ctas, cudaStream_t s)
{
    fdtd_grid* g = const_cast<fdtd_grid*>(cg);
    if (g->desc.precision != FDTD_F32 || needs_cell_passes(g)) return cudaErrorInvalidValue;
    constexpr int RY = 16;
    using S = Tb2Smem<RY>;
    int per_sm = 0;
    cudaError_t e = tb2_blocks_per_sm<RY>(&per_sm);
    if (e != cudaSuccess) return e;
    const int all = std::min(kTb2MaxCtas, (g->sm_count > 0 ? g->sm_count : 152) * per_sm);
    const int slots = std::max(1, std::min(all, max_ctas));
    TileConfig tc = g->tile;
    Tb2Plan plan;
    tb2_plan(g, RY, slots, tc, plan);
    yee_tb2_t<RY><<<unsigned(slots), dim3(32, RY), S::bytes(), s>>>(make_args<float>(g, cur), times, i0, i1, plan);
    return cudaGetLastError();
}

}  // namespace fdtd

using namespace fdtd;

extern "C" {

int fdtd_debug_tb2_order(int t, int u, int nz, int slots, int order, int* out)
{
    if (t < 1 || u < 1 || nz < 1 || slots < 1 || !out) return -1;
    const int D = tb2_order_d(t, u, nz, slots, order == 2 ? 2 : 1);
    for (int m = 0; m < t * u; ++m) out[m] = tb2_window_host(t, u, D, m);
    return D;
}

fdtd_status fdtd_debug_tb2_refine(int slots, const long long* starts, const unsigned long long* cycles, double step,
                                  long long* out)
{
    if (slots < 1 || !starts || !cycles || !out || !(step > 0.0 && step <= 1.0))
        return fail(FDTD_EINVAL, "invalid argument");
    std::vector<long long> s(starts, starts + slots + 1);
    if (s[0] != 0) return fail(FDTD_EINVAL, "starts[0] must be 0");
    for (int c = 0; c < slots; ++c)
        if (s[size_t(c) + 1] < s[size_t(c)]) return fail(FDTD_EINVAL, "starts must not decrease");
    const std::vector<long long> ns = tb2_refined_ranges(s, cycles, step);
    for (int c = 0; c <= slots; ++c) out[c] = ns[size_t(c)];
    return FDTD_OK;
}

}  // extern "C"
