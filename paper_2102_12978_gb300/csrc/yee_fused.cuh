// yee_fused.cuh -- one full Yee step per launch, fused with the CPML, the
// Bessel-antenna soft source and the fluence (Section 4, Eq. 13, Section 2).
//
// Work decomposition (sm_103a, HBM-bound stencil, no tensor-core contraction):
//   * A CTA of TX x TY threads owns a TX x TY tile of (i, j) columns and one
//     z-segment [kb, ke); every thread owns one column and marches along z.
//   * E^n planes pass through a 4-slot shared-memory ring covering the tile
//     plus a one-cell halo on every side; each thread prefetches its own (and
//     one halo) cell of plane k+2 into registers while plane k is computed.
//   * H^{n+1/2} of plane k is computed on the tile plus a one-cell low halo
//     (column i0-1, row j0-1), so that E^{n+1} of plane k, which needs
//     H^{n+1/2}(i-1), (j-1), (k-1), is finished in the same pass.  Reading
//     step n from one copy of the fields and writing step n+1 into the other
//     (ping-pong) makes the halo recompute race-free.
//   * The fluence term of step n, |E^n x (H^{n-1/2}+H^{n+1/2})/2| dt at the
//     centre of cell (i-1, j-1, k-1), uses the E^n ring and a two-plane ring of
//     H-bar in shared memory; the last tile of each axis also takes the cell
//     next to the virtual PEC wall.
//   * CPML psi (Roden-Gedney) lives in compact shell arrays: H-side psi is
//     ping-ponged (the halo recompute reads it), E-side psi is updated in place.
//   * The soft source (Eq. 13) reads an antenna mask per column and an FP64
//     complex coefficient per (component, column); the time factor
//     e^{-i omega t'} f(t) is evaluated once per CTA in FP64 and the phase
//     along z comes from an FP64 table e^{i beta z_k}.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fdtd {

struct SrcTime {
    int gauss;          // 0: CW with sin^2 ramp, 1: Gaussian
    double ramp, T, T0;
    double dt;
};

template <typename real>
struct StepArgs {
    int nx, ny, nz, npml, pitch;
    const real* ein[3];
    real* eout[3];
    const real* hin[3];
    real* hout[3];
    const real* phx_in[2];   // x shell H psi: Hyx, Hzx   [k][j][2 npml]
    real* phx_out[2];
    const real* phy_in[2];   // y shell H psi: Hxy, Hzy   [k][2 npml][pitch]
    real* phy_out[2];
    real* pex[2];            // x shell E psi: Eyx, Ezx (in place)
    real* pey[2];            // y shell E psi: Exy, Ezy (in place)
    real* pex_out[2];        // the other copy of the E psi: the two-step kernel reads
    real* pey_out[2];        // pex / pey and writes here (ping-pong)
    const real* chx;         // dt / (kappa dx) at H x-positions (i+1/2), length nx
    const real* chy;         // dt / (kappa dy) at H y-positions (j+1/2), length ny
    const real* cex;         // dt / (kappa dx) at E x-positions i
    const real* cey;
    const real* bhx;         // CPML b and a' = dt a / d on the shells, length 2 npml
    const real* ahx;
    const real* bex;
    const real* aex;
    const real* bhy;
    const real* ahy;
    const real* bey;
    const real* aey;
    real cz;                 // dt / dz
    double dt;
    double dt16;             // dt / 16: the fluence term's factor (the 1/16 of its centre means folded in)
    void* fluence;           // [nz][ny][pitch] accumulator or null: double (FP64
                             // grids) or float2 (sum, Kahan compensation) (FP32)
    const uint8_t* smask;    // [ny][nx] or null (no source)
    const double2* scoef;    // [6][ny][nx]  FP64 antenna coefficients
    const void* scoefr;      // the same in the field precision (float2 / double2)
    const double2* zph;      // [nz]: e^{i beta k dz} (coefficients carry the half-cell z offset)
    const void* zphr;        // the same in the field precision (float2 / double2)
    SrcTime st;
    int fault;               // test hook (fdtd_debug_inject_fault): 1 = CTA (0,0,0) withholds one plane's copies
    // z walls (Section 2's Bessel-Gauss box; the cell passes only): PEC at
    // z = 0 and z = nz dz, npz CPML cells inside each
    int zw, npz;
    const real* phz_in[2];   // z shell H psi: Hxz, Hyz   [2 npz][ny][pitch]
    real* phz_out[2];
    real* pez[2];            // z shell E psi: Exz, Eyz (in place)
    const real* chz;         // dt / (kappa dz) at H z-positions (k+1/2), length nz
    const real* cez;         // dt / (kappa dz) at E z-positions k
    const real* bhz;         // CPML b and a' = dt a / dz on the z shell, length 2 npz
    const real* ahz;
    const real* bez;
    const real* aez;
    // wall source (Section 2): E_x on plane wplane += Re{ W[col] tw }
    const void* wcoefr;      // [ny][nx] in the field precision, or null
    int wplane;
    // cell passes: plane of blockIdx.z = 0 (grids of more than 65535 planes
    // are launched in chunks of planes)
    int kbase;
};

// Time factor of the soft source at time t: cos / sin of the phase
// 2 pi frac(t') (t' = t, or t - T0 for the Gaussian) and the envelope f.
// Host and device evaluate it in FP64.
__host__ __device__ __forceinline__ void source_time(const SrcTime& st, double t, double& c, double& s,
                                                     double& f)
{
    double tp = st.gauss ? t - st.T0 : t;
    double ph = 2.0 * 3.14159265358979323846 * (tp - floor(tp));
#ifdef __CUDA_ARCH__
    sincos(ph, &s, &c);
#else
    s = sin(ph);
    c = cos(ph);
#endif
    if (st.gauss) {
        double u = (t - st.T0) / st.T;
        f = exp(-u * u);
    } else if (t < st.ramp) {
        double sn = sin(3.14159265358979323846 * t / (2.0 * st.ramp));
        f = sn * sn;
    } else {
        f = 1.0;
    }
}

// Fluence accumulator of one cell.  FP64 grids add in FP64.  FP32 grids keep
// an FP32 sum with a Kahan compensation term (no FP64 instruction per cell:
// GB300's FP64 pipe is a small fraction of its FP32 rate).
template <typename real> struct FluAcc;
template <> struct FluAcc<double> {
    using T = double;
    __device__ __forceinline__ static T add(T old, double v_dt) { return old + v_dt; }
};
template <> struct FluAcc<float> {
    using T = float2;
    __device__ __forceinline__ static T add(T old, float v_dt)
    {
        const float y = v_dt - old.y;
        const float t = old.x + y;
        return make_float2(t, (t - old.x) - y);
    }
};

// Value added by the soft source: f Re{ B e^{i beta z} e^{-i Phi} }.
__device__ __forceinline__ double source_value(double2 B, double2 z, double c, double s, double f)
{
    double ur = z.x * c + z.y * s;
    double ui = z.y * c - z.x * s;
    return f * (B.x * ur - B.y * ui);
}

template <typename real, int TX, int TY>
struct FusedTile {
    static constexpr int PX = TX + 2;
    static constexpr int PY = TY + 2;
    static constexpr int P = PX * PY;
    static constexpr int NT = TX * TY;
    static constexpr int NHE = 2 * PX + 2 * TY;   // halo cells of the E ring
    static constexpr int NHH = TX + TY + 1;       // halo cells of the H recompute
    static constexpr size_t smem_bytes() { return size_t(4 * 3 + 2 * 3 + 2 * 3) * P * sizeof(real); }
};

template <typename real, int TX, int TY>
__global__ void __launch_bounds__(TX * TY)
yee_step_fused(const StepArgs<real> a, long long n, int lz)
{
    using T = FusedTile<real, TX, TY>;
    constexpr int PX = T::PX, P = T::P, NT = T::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real* sE = reinterpret_cast<real*>(smem_raw);   // [4][3][P]
    real* sH = sE + 12 * P;                          // [2][3][P]
    real* sB = sH + 6 * P;                           // [2][3][P]
    __shared__ double tf[6];

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const int kb = blockIdx.z * lz;
    const int ke = min(kb + lz, a.nz);
    const int nx = a.nx, ny = a.ny, nz = a.nz, pitch = a.pitch, npml = a.npml;
    const size_t plane = size_t(pitch) * ny;
    const int i = i0 + tx, j = j0 + ty;
    const bool own = (i < nx) && (j < ny);
    const int so = (ty + 1) * PX + (tx + 1);   // own cell in the smem tile

    if (tid == 0) {
        double c, s, f;
        source_time(a.st, (double(n) + 0.5) * a.dt, c, s, f);
        tf[3] = c; tf[4] = s; tf[5] = f;
        source_time(a.st, (double(n) + 1.0) * a.dt, c, s, f);
        tf[0] = c; tf[1] = s; tf[2] = f;
    }
    for (int q = tid; q < 12 * P; q += NT) { sH[q] = real(0); }   // sH and sB

    // ---- E^n ring loader: own cell + one halo cell per thread (tid < NHE)
    static_assert(T::NHE <= NT && T::NHH <= NT, "tile too small for its halo");
    const bool has_he = tid < T::NHE;
    int hi_e = -1, hj_e = -1, hs_e = 0;
    if (has_he) {
        int ii, jj;
        if (tid < PX) { ii = tid; jj = 0; }
        else if (tid < 2 * PX) { ii = tid - PX; jj = T::PY - 1; }
        else if (tid < 2 * PX + TY) { ii = 0; jj = 1 + tid - 2 * PX; }
        else { ii = PX - 1; jj = 1 + tid - 2 * PX - TY; }
        hi_e = i0 - 1 + ii; hj_e = j0 - 1 + jj; hs_e = jj * PX + ii;
    }
    const bool halo_e_in = hi_e >= 0 && hi_e < nx && hj_e >= 0 && hj_e < ny;
    real pe[3], peh[3];
    auto fetch_e = [&](int kp) {
        int kw = kp % nz; if (kw < 0) kw += nz;
        size_t base = size_t(kw) * plane;
        #pragma unroll
        for (int c = 0; c < 3; ++c) {
            pe[c] = own ? a.ein[c][base + size_t(j) * pitch + i] : real(0);
            peh[c] = halo_e_in ? a.ein[c][base + size_t(hj_e) * pitch + hi_e] : real(0);
        }
    };
    auto commit_e = [&](int kp) {
        real* s = sE + (kp & 3) * 3 * P;
        #pragma unroll
        for (int c = 0; c < 3; ++c) {
            s[c * P + so] = pe[c];
            if (has_he) s[c * P + hs_e] = peh[c];
        }
    };

    // ---- H halo cell of this thread (tid < NHH)
    int hi_h = -1, hj_h = -1, hs_h = 0;
    if (tid < T::NHH) {
        if (tid < TX) { hi_h = i0 + tid; hj_h = j0 - 1; hs_h = tid + 1; }
        else { hi_h = i0 - 1; hj_h = j0 - 1 + (tid - TX); hs_h = (tid - TX) * PX; }
    }
    const bool halo_h_in = hi_h >= 0 && hi_h < nx && hj_h >= 0 && hj_h < ny;

    real ph[3], phh[3];
    auto fetch_h = [&](int kp) {
        int kw = kp % nz; if (kw < 0) kw += nz;
        size_t base = size_t(kw) * plane;
        #pragma unroll
        for (int c = 0; c < 3; ++c) {
            ph[c] = own ? a.hin[c][base + size_t(j) * pitch + i] : real(0);
            phh[c] = halo_h_in ? a.hin[c][base + size_t(hj_h) * pitch + hi_h] : real(0);
        }
    };

    // H^{n+1/2} at (ci, cj, plane kp) from the E ring; writes psi if `store`.
    auto compute_h = [&](int ci, int cj, int kp, int sidx, const real hold[3], bool store,
                         uint8_t mk, real chx, real chy, real hnew[3]) {
        int kw = kp % nz; if (kw < 0) kw += nz;
        const real* e0 = sE + (kp & 3) * 3 * P;
        const real* e1 = sE + ((kp + 1) & 3) * 3 * P;
        real ex = e0[sidx], ey = e0[P + sidx], ez = e0[2 * P + sidx];
        real dEz_y = e0[2 * P + sidx + PX] - ez;
        real dEy_z = e1[P + sidx] - ey;
        real dEx_z = e1[sidx] - ex;
        real dEz_x = e0[2 * P + sidx + 1] - ez;
        real dEy_x = e0[P + sidx + 1] - ey;
        real dEx_y = e0[sidx + PX] - ex;
        real hx = hold[0] - chy * dEz_y + a.cz * dEy_z;
        real hy = hold[1] - a.cz * dEx_z + chx * dEz_x;
        real hz = hold[2] - chx * dEy_x + chy * dEx_y;
        if (npml > 0) {
            const int w2 = 2 * npml;
            if (ci < npml || ci >= nx - npml) {
                int ii = ci < npml ? ci : ci - nx + w2;
                size_t q = (size_t(kw) * ny + cj) * w2 + ii;
                real b = a.bhx[ii], aa = a.ahx[ii];
                real p0 = b * a.phx_in[0][q] + aa * dEz_x;     // Hyx
                real p1 = b * a.phx_in[1][q] + aa * dEy_x;     // Hzx
                hy += p0;
                hz -= p1;
                if (store) { a.phx_out[0][q] = p0; a.phx_out[1][q] = p1; }
            }
            if (cj < npml || cj >= ny - npml) {
                int jj = cj < npml ? cj : cj - ny + w2;
                size_t q = (size_t(kw) * w2 + jj) * pitch + ci;
                real b = a.bhy[jj], aa = a.ahy[jj];
                real p0 = b * a.phy_in[0][q] + aa * dEz_y;     // Hxy
                real p1 = b * a.phy_in[1][q] + aa * dEx_y;     // Hzy
                hx -= p0;
                hz += p1;
                if (store) { a.phy_out[0][q] = p0; a.phy_out[1][q] = p1; }
            }
        }
        {
            if (mk & 0x38) {
                const size_t ncol = size_t(nx) * ny, col = size_t(cj) * nx + ci;
                double c = tf[3], s = tf[4], f = tf[5];
                if (mk & 0x08) hx += real(source_value(a.scoef[3 * ncol + col], a.zph[kw], c, s, f));
                if (mk & 0x10) hy += real(source_value(a.scoef[4 * ncol + col], a.zph[kw], c, s, f));
                if (mk & 0x20) hz += real(source_value(a.scoef[5 * ncol + col], a.zph[kw], c, s, f));
            }
        }
        hnew[0] = hx; hnew[1] = hy; hnew[2] = hz;
    };

    // per-column constants of the own and the halo-H cell
    const uint8_t mk_own = (own && a.smask) ? a.smask[size_t(j) * nx + i] : uint8_t(0);
    const uint8_t mk_hh = (halo_h_in && a.smask) ? a.smask[size_t(hj_h) * nx + hi_h] : uint8_t(0);
    const real chx_o = own ? a.chx[i] : real(0), chy_o = own ? a.chy[j] : real(0);
    const real cex_o = own ? a.cex[i] : real(0), cey_o = own ? a.cey[j] : real(0);
    const real chx_h = halo_h_in ? a.chx[hi_h] : real(0), chy_h = halo_h_in ? a.chy[hj_h] : real(0);

    // ---- prologue
    fetch_e(kb - 1);
    commit_e(kb - 1);
    fetch_e(kb);
    fetch_h(kb - 1);
    const bool do_flu = a.fluence != nullptr;

    for (int k = kb - 1; k <= ke; ++k) {
        commit_e(k + 1);
        real hold[3] = {ph[0], ph[1], ph[2]};
        real hold_h[3] = {phh[0], phh[1], phh[2]};
        if (k + 2 <= ke + 1) fetch_e(k + 2);
        if (k + 1 <= ke) fetch_h(k + 1);
        __syncthreads();   // A: E planes k, k+1 visible; previous readers done

        const int kw = ((k % nz) + nz) % nz;
        const bool write_k = (k >= kb) && (k < ke);
        real* hs = sH + (k & 1) * 3 * P;
        real* bs = sB + (k & 1) * 3 * P;
        if (own) {
            real hn[3];
            compute_h(i, j, k, so, hold, write_k, mk_own, chx_o, chy_o, hn);
            #pragma unroll
            for (int c = 0; c < 3; ++c) {
                hs[c * P + so] = hn[c];
                bs[c * P + so] = real(0.5) * (hold[c] + hn[c]);
            }
            if (write_k) {
                size_t g = size_t(kw) * plane + size_t(j) * pitch + i;
                #pragma unroll
                for (int c = 0; c < 3; ++c) a.hout[c][g] = hn[c];
            }
        } else {
            #pragma unroll
            for (int c = 0; c < 3; ++c) { hs[c * P + so] = real(0); bs[c * P + so] = real(0); }
        }
        if (tid < T::NHH) {
            if (halo_h_in) {
                real hn[3];
                compute_h(hi_h, hj_h, k, hs_h, hold_h, false, mk_hh, chx_h, chy_h, hn);
                #pragma unroll
                for (int c = 0; c < 3; ++c) {
                    hs[c * P + hs_h] = hn[c];
                    bs[c * P + hs_h] = real(0.5) * (hold_h[c] + hn[c]);
                }
            } else {
                #pragma unroll
                for (int c = 0; c < 3; ++c) { hs[c * P + hs_h] = real(0); bs[c * P + hs_h] = real(0); }
            }
        }
        __syncthreads();   // B: H^{n+1/2} planes k, k-1 and H-bar visible

        if (write_k && own) {
            const real* h0 = sH + (k & 1) * 3 * P;
            const real* h1 = sH + ((k - 1) & 1) * 3 * P;
            const real* e0 = sE + (k & 3) * 3 * P;
            real ex = e0[so], ey = e0[P + so], ez = e0[2 * P + so];
            real hx0 = h0[so], hy0 = h0[P + so], hz0 = h0[2 * P + so];
            real dHz_y = hz0 - h0[2 * P + so - PX];
            real dHy_z = hy0 - h1[P + so];
            real dHx_z = hx0 - h1[so];
            real dHz_x = hz0 - h0[2 * P + so - 1];
            real dHy_x = hy0 - h0[P + so - 1];
            real dHx_y = hx0 - h0[so - PX];
            const real cey = cey_o, cex = cex_o;
            real nex = ex + cey * dHz_y - a.cz * dHy_z;
            real ney = ey + a.cz * dHx_z - cex * dHz_x;
            real nez = ez + cex * dHy_x - cey * dHx_y;
            if (npml > 0) {
                const int w2 = 2 * npml;
                if (i < npml || i >= nx - npml) {
                    int ii = i < npml ? i : i - nx + w2;
                    size_t q = (size_t(kw) * ny + j) * w2 + ii;
                    real b = a.bex[ii], aa = a.aex[ii];
                    real p0 = b * a.pex[0][q] + aa * dHz_x;     // Eyx
                    real p1 = b * a.pex[1][q] + aa * dHy_x;     // Ezx
                    a.pex[0][q] = p0; a.pex[1][q] = p1;
                    ney -= p0;
                    nez += p1;
                }
                if (j < npml || j >= ny - npml) {
                    int jj = j < npml ? j : j - ny + w2;
                    size_t q = (size_t(kw) * w2 + jj) * pitch + i;
                    real b = a.bey[jj], aa = a.aey[jj];
                    real p0 = b * a.pey[0][q] + aa * dHz_y;     // Exy
                    real p1 = b * a.pey[1][q] + aa * dHx_y;     // Ezy
                    a.pey[0][q] = p0; a.pey[1][q] = p1;
                    nex += p0;
                    nez -= p1;
                }
            }
            {
                const uint8_t mk = mk_own;
                if (mk & 0x07) {
                    const size_t ncol = size_t(nx) * ny, col = size_t(j) * nx + i;
                    double c = tf[0], s = tf[1], f = tf[2];
                    if (mk & 0x01) nex += real(source_value(a.scoef[col], a.zph[kw], c, s, f));
                    if (mk & 0x02) ney += real(source_value(a.scoef[ncol + col], a.zph[kw], c, s, f));
                    if (mk & 0x04) nez += real(source_value(a.scoef[2 * ncol + col], a.zph[kw], c, s, f));
                }
            }
            if (j == 0) { nex = real(0); nez = real(0); }    // PEC, tangential E
            if (i == 0) { ney = real(0); nez = real(0); }
            size_t g = size_t(kw) * plane + size_t(j) * pitch + i;
            a.eout[0][g] = nex; a.eout[1][g] = ney; a.eout[2][g] = nez;
        }

        if (do_flu && k >= kb + 1) {
            // cells (fi, fj, k-1) with fi in {i-1, i at the +x wall}, fj likewise
            const int km = k - 1;
            const int kmw = ((km % nz) + nz) % nz;
            const real* em = sE + (km & 3) * 3 * P;
            const real* ek = sE + (k & 3) * 3 * P;
            const real* bm = sB + (km & 1) * 3 * P;
            const real* bk = sB + (k & 1) * 3 * P;
            const bool xw = (tx == TX - 1) && (i == nx - 1) && (j <= ny);
            const bool yw = (ty == TY - 1) && (j == ny - 1) && (i <= nx);
            #pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int di = q & 1, dj = q >> 1;
                if (di && !xw) continue;
                if (dj && !yw) continue;
                const int fi = i - 1 + di, fj = j - 1 + dj;
                if (fi < 0 || fj < 0 || fi >= nx || fj >= ny) continue;
                const int sc = so - PX - 1 + dj * PX + di;   // smem index of (fi, fj)
                real ex = real(0.25) * (em[sc] + em[sc + PX] + ek[sc] + ek[sc + PX]);
                real ey = real(0.25) * (em[P + sc] + em[P + sc + 1] + ek[P + sc] + ek[P + sc + 1]);
                real ez = real(0.25) * (em[2 * P + sc] + em[2 * P + sc + 1] + em[2 * P + sc + PX] +
                                        em[2 * P + sc + PX + 1]);
                real hx = real(0.5) * (bm[sc] + bm[sc + 1]);
                real hy = real(0.5) * (bm[P + sc] + bm[P + sc + PX]);
                real hz = real(0.5) * (bm[2 * P + sc] + bk[2 * P + sc]);
                real sx = ey * hz - ez * hy;
                real sy = ez * hx - ex * hz;
                real sz = ex * hy - ey * hx;
                real sm = sqrt(sx * sx + sy * sy + sz * sz);
                size_t g = size_t(kmw) * plane + size_t(fj) * pitch + fi;
                using Acc = FluAcc<real>;
                typename Acc::T* F = static_cast<typename Acc::T*>(a.fluence);
                F[g] = Acc::add(F[g], sm * real(a.dt));
            }
        }
    }
}

}  // namespace fdtd
