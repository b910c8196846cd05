// yee_tb2.cuh -- two Yee steps per launch (temporal blocking), FP32 (sm_103a).
//
// One launch advances the grid from (E^n, H^{n-1/2}) to (E^{n+2}, H^{n+3/2})
// and adds the fluence terms of steps n and n+1, so that the fields, the
// fluence accumulator and the CPML psi cross HBM once per two steps: half the
// bytes per cell-update of any one-step pass.  Every arithmetic step is the
// one of the cell passes (Section 4 Yee update with the Roden-Gedney CPML,
// the soft source of Eq. 13, the fluence of Section 2), in the same order.
//
// Work decomposition.
//   * A CTA of 32 x RY threads owns a window of 32 x RY (i, j) columns; each
//     thread owns one column and marches along z.  Windows overlap by two
//     columns / rows on each side: a window updates E^{n+2} only on its inner
//     28 x (RY - 4) columns (windows on the box faces also on the face side,
//     where the PEC wall supplies the neighbours), and recomputes the two
//     outer rings itself (H^{n+1/2} on the window less its last column,
//     E^{n+1} one column in, H^{n+3/2} another).  Columns past the box hold
//     exact zeros at every stage (zero-filled loads, zero coefficients): the
//     wall values the stencil reads there.
//   * z-march with a wavefront of four stages per plane p: A, H^{n+1/2} of
//     plane p-1; B, E^{n+1} of plane p-1; C, H^{n+3/2} of plane p-2; D,
//     E^{n+2} of plane p-2.  The +x / -x neighbours come from the adjacent
//     lane by warp shuffle, the +y / -y neighbours from per-plane shared
//     exchange buffers (two CTA barriers per plane), the +z / -z neighbours
//     from registers carried from plane to plane.
//   * Each thread streams its own column: the E^n and H^{n-1/2} values and
//     the fluence accumulator of plane p + 3 and the CPML psi of plane p + 2
//     (shell columns) are copied by cp.async (zero-filled past the box) into
//     a per-thread ring of four plane slots in shared memory (see
//     tb2_issue); a thread waits only for its
//     own copies, so the ring needs no barrier.  The psi of a plane are
//     updated in place in its slot (n-1/2 -> n+1/2, n -> n+1) and read back
//     by the second step's stages.  The plane loop is unrolled by two, so
//     the exchange buffers' parities are constants; the ring slot is an index
//     (a four-fold unroll that made it a constant too ran 1 % slower: its
//     loop body is twice as large).
//   * The antenna coefficients of a window's columns are staged in shared
//     memory when the window starts; the per-plane phase e^{i beta z_k} is
//     loaded one plane ahead.
//   * The fluence of cell (i, j, k) needs E and H at i+1, j+1, k+1; a
//     window's fluence cells are its E^{n+2} cells shifted by -1 in x, y and
//     z (plus the last cell before the far wall), so that the H^{n+3/2} they
//     need lie inside the window.  Both terms of a cell (steps n and n+1) are
//     added, Kahan-compensated, in one read-modify-write.
//   * Reading step n from one copy of the fields and psi and writing step
//     n+2 into the other (ping-pong, E-side psi included) makes the halo
//     recompute race-free.
//   * Every row of a window runs every stage, whether or not a column the
//     window writes depends on it, so that the stage code has no branches
//     on the row; a row with antenna points adds the source terms on all its
//     lanes (zero terms where a column has none), and the x-shell windows
//     update the x psi on all lanes (zero coefficients off the shell).
//     Windows off the box faces and the CPML shells run code without the
//     checks of the walls, psi and columns past the box (template flags GX,
//     GY).
//   * A CTA takes a contiguous range of the flattened (window, plane) work:
//     ranges of equal estimated cost (windows with CPML shell or antenna
//     columns weigh more, with weights the autotuner picks by timing), or
//     ranges the host refined until the CTAs' measured times were equal
//     (the kernel records each CTA's SM cycles when asked).  The window rows
//     may be interleaved in the flattened order, so that x-neighbouring
//     windows march side by side (tb2_window_at).  Where a range starts or
//     crosses into the next window the wavefront restarts, which costs three
//     planes of recompute.
//   * Outputs are stored with the L2 evict-last policy; every sum of two
//     products is rounded explicitly (see below).
// z-periodic grids only (the antenna boxes of Section 4); FP32 fields with the
// Kahan FP32 fluence.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "yee_cell.cuh"

namespace fdtd {

// Source time factors f e^{-i Phi} of the two steps: H at (n+1/2) dt and
// (n+3/2) dt, E at (n+1) dt and (n+2) dt.
struct Tb2Times {
    Cpx<float> th0, te0, th1, te1;
};

// Flattened work: windows T (along x) by U (along y), nz planes each, items
// (window, plane) numbered window * nz + plane.  CTA c takes the items
// [start[c], start[c + 1]): ranges of equal estimated cost (a window's planes
// cost more where the window holds CPML shell or antenna columns), chosen on
// the host.
// prof, if not null, receives per CTA c the SM cycles it ran (prof[c] is
// added to): the host moves the ranges' boundaries so that every CTA takes
// the same time.
constexpr int kTb2MaxCtas = 512;
// D > 1: the windows of D window rows are interleaved in the flattened
// order (position item / nz): group g of rows gD .. gD + D - 1 (fewer in the
// last group) takes the positions from g T D on, window (wx, gD + l) at
// position g T D + wx * (rows in the group) + l, so that x-neighbours lie D
// positions apart.  The host picks D so that D windows of planes are close to
// a whole number of CTA shares: x-neighbours then start at nearly the same
// plane and march side by side.  D = 1: row by row.
struct Tb2Plan {
    int T, U, D;
    unsigned long long* prof;
    long long start[kTb2MaxCtas + 1];
};

__device__ __forceinline__ int tb2_window_at(const Tb2Plan& tw, int pos)
{
    if (tw.D <= 1) return pos;
    const int grp = pos / (tw.T * tw.D);
    const int rows = tw.U - grp * tw.D < tw.D ? tw.U - grp * tw.D : tw.D;
    const int r = pos - grp * tw.T * tw.D;
    const int wx = r / rows, l = r - wx * rows;
    return (grp * tw.D + l) * tw.T + wx;
}

// Columns per window along x, and the stride between windows.
constexpr int kTb2Wx = 32;
constexpr int kTb2Sx = 28;


template <int RY>
struct Tb2Smem {
    static constexpr int NT = 32 * RY;   // threads (columns) per window
    static constexpr int R = 4;          // ring slots per thread (see tb2_issue)
    static constexpr int NF = 14;        // ring floats per slot: E^n 3, H^{n-1/2} 3, psi 8
    // exchange arrays: a row of zeros before and after the window's RY rows
    // (the values of the rows beyond it), so that a y neighbour is one plain
    // shared load; thread tid's value at XO + tid.  Consecutive arrays share
    // a zero row (the row after array a is the row before array a + 1), and
    // one more zero row follows the last array.
    static constexpr int XS = NT + 32, XO = 32;
    static constexpr int NX = 14;         // 2x2 E^n, 3 H^{n+1/2}, 2x2 E^{n+1}, 3 H^{n+3/2}
    static constexpr size_t bytes()
    {
        return size_t(R) * NT * 8                 // fluence accumulator (float2) per slot
               + size_t(R) * NF * NT * 4          // fields and psi per slot
               + (size_t(NX) * XS + 32) * 4       // exchange arrays and their zero rows
               + size_t(12) * NT * 4;             // antenna coefficients of the column (6 complex)
    }
};

__device__ __forceinline__ void cpa4(float* dst, const float* src, bool valid)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cpa8(float2* dst, const float2* src, bool valid)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(valid ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cpa_wait2() { asm volatile("cp.async.wait_group 2;" ::: "memory"); }
__device__ __forceinline__ void cpa_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Every sum of two products below is written with explicit roundings
// (mul_rn / fma_rn): the plane loop runs two instantiations of tb2_plane
// (the exchange parities), and which one computes a plane depends on where
// the CTA's range of planes starts; left to the compiler, the two could
// contract such a sum into a fused multiply-add in different ways, and the
// results would depend on the CTAs' work split.

// |E x Hbar| dt of a cell from its centre sums (the 1/16 of the four-edge E
// means and the two-face, two-time H means is folded into dt16).
__device__ __forceinline__ float tb2_flux(float cx, float cy, float cc, float hbx, float hby, float hbz, float dt16)
{
    const float sx = fma_rn(cy, hbz, -mul_rn(cc, hby));
    const float sy = fma_rn(cc, hbx, -mul_rn(cx, hbz));
    const float sz = fma_rn(cx, hby, -mul_rn(cy, hbx));
    return mul_rn(vec_norm(fma_rn(sz, sz, fma_rn(sy, sy, mul_rn(sx, sx)))), dt16);
}

__device__ __forceinline__ Cpx<float> cmul(Cpx<float> z, Cpx<float> t)
{
    return Cpx<float>{fma_rn(z.x, t.x, -mul_rn(z.y, t.y)), fma_rn(z.x, t.y, mul_rn(z.y, t.x))};
}

// Stores of the window's outputs with the L2 evict-last priority: a window
// writes its own 28 columns of a row, so the first and last 32-byte sectors
// of the row are shared with the neighbouring windows, which write their
// part at another time; kept in L2 until the neighbour's part arrives, such
// a sector reaches DRAM whole.
__device__ __forceinline__ uint64_t tb2_store_policy()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void st_keep(float* q, float v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(q), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_keep(float2* q, float2 v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(q), "f"(v.x), "f"(v.y), "l"(pol)
                 : "memory");
}

// CPML psi update b psi + a d.
__device__ __forceinline__ float psi_rn(float b, float psi, float aa, float d) { return fma_rn(b, psi, mul_rn(aa, d)); }

// Per-window constants of a thread's column.
struct Tb2Col {
    int i, j, lane, row, tid;
    bool indom, own, fown, sx, sy, ant;   // ant: the window holds antenna columns
    bool anth, ante;                      // warp-uniform: the row holds antenna H / E points
    uint8_t mk;
    int col, colx, coly;
    float chx, chy, cex, cey, bhx, ahx, bex, aex, bhy, ahy, bey, aey;
};

// Values carried from plane to plane (planes relative to the current p).
struct Tb2Carry {
    float e0[3];                  // E^n(p-1)
    float h1p[3];                 // H^{n+1/2}(p-2)
    float e1p[3];                 // E^{n+1}(p-2)
    float h2px, h2py;             // H^{n+3/2}(p-3), x and y
    // fluence centre sums: step n of plane p-2 (f), step n+1 of plane p-3 (g)
    float fPEx, fPEy, fcz, fhbx, fhby, fHsz;
    float gPEx, gPEy, gcz, ghbx, ghby, gHsz;
    float tn;                     // fluence term of step n, plane p-3
    int kp, kq, kr, k3, ki;       // planes of p, p-1, p-2, p-3 and p+2 (modulo nz)
    Cpx<float> zq, zr;            // e^{i beta z} of planes p-1 and p-2
};

template <int RY>
struct Tb2Bufs {
    float2* fring;   // [R][NT]
    float* ring;     // [R][NF][NT]
    float* EB;       // [2][Ez, Ex][XS]: E^n of a plane
    float* HB;       // [Hx, Hz, Hy^{n-1/2} + Hy^{n+1/2}][XS]
    float* E1B;      // [2][Ez, Ex][XS]: E^{n+1}
    float* H1B;      // [Hx, Hz, Hy^{n+1/2} + Hy^{n+3/2}][XS]
    float2* SC;      // [6][NT]: antenna coefficients (zero where a column has no point of the component)
};

__device__ __forceinline__ int next_plane(int k, int nz) { return k + 1 == nz ? 0 : k + 1; }

// Copies of this thread's column, one cp.async group: E^n and H^{n-1/2} of
// plane k and the fluence accumulator of plane kf into slot s, the psi of
// plane kp into slot sp.  A plane's fields are first read at its own stage A
// (E^n) and its psi one plane later (stage A of the next plane), so that at
// the end of plane p the fields of p + 3 (fluence p) go into the slot the
// fields of p - 1 have left and the psi of p + 2 into the slot the psi of
// p - 2 have left: with four slots the fields are copied three planes ahead
// of their first use, the psi two and a half.
template <int RY, int G>
__device__ __forceinline__ void tb2_issue(const StepArgs<float>& a, const Tb2Col& c, const Tb2Bufs<RY>& b, int s,
                                          int k, int kf, int sp, int kp)
{
    using S = Tb2Smem<RY>;
    constexpr int NT = S::NT, NF = S::NF;
    float* r = b.ring + s * NF * NT + c.tid;
    float* rs = b.ring + sp * NF * NT + c.tid;
    constexpr bool GX = G & 1, GY = G & 2;
    const int g = k * (a.pitch * a.ny) + c.col;
    cpa4(r + 0 * NT, a.ein[0] + g, (!GX && !GY) || c.indom);
    cpa4(r + 1 * NT, a.ein[1] + g, (!GX && !GY) || c.indom);
    cpa4(r + 2 * NT, a.ein[2] + g, (!GX && !GY) || c.indom);
    cpa4(r + 3 * NT, a.hin[0] + g, (!GX && !GY) || c.indom);
    cpa4(r + 4 * NT, a.hin[1] + g, (!GX && !GY) || c.indom);
    cpa4(r + 5 * NT, a.hin[2] + g, (!GX && !GY) || c.indom);
    if (GX) {   // every lane: zeros where the column is not in an x shell
        const int q = kp * a.ny * (2 * a.npml) + c.colx;
        cpa4(rs + 6 * NT, a.phx_in[0] + q, c.sx);    // Hyx
        cpa4(rs + 7 * NT, a.phx_in[1] + q, c.sx);    // Hzx
        cpa4(rs + 10 * NT, a.pex[0] + q, c.sx);      // Eyx
        cpa4(rs + 11 * NT, a.pex[1] + q, c.sx);      // Ezx
    }
    if (GY && c.sy) {
        const int q = kp * (2 * a.npml) * a.pitch + c.coly;
        cpa4(rs + 8 * NT, a.phy_in[0] + q, true);    // Hxy
        cpa4(rs + 9 * NT, a.phy_in[1] + q, true);    // Hzy
        cpa4(rs + 12 * NT, a.pey[0] + q, true);      // Exy
        cpa4(rs + 13 * NT, a.pey[1] + q, true);      // Ezy
    }
    const float2* F = static_cast<const float2*>(a.fluence);
    cpa8(b.fring + s * NT + c.tid, c.fown ? F + kf * (a.pitch * a.ny) + c.col : reinterpret_cast<const float2*>(a.ein[0]),
         c.fown);
    cpa_commit();
}

// Soft-source increment Re{coef_c u} of component comp (coefficients staged in
// SC; zero, and the increment a signed zero, where the column has no point of
// the component).
template <int RY>
__device__ __forceinline__ float tb2_src(const Tb2Bufs<RY>& b, const Tb2Col& c, int comp, Cpx<float> u)
{
    constexpr int NT = Tb2Smem<RY>::NT;
    const float2 v = b.SC[comp * NT + c.tid];
    return fma_rn(v.x, u.x, -mul_rn(v.y, u.y));
}

// One plane p of the wavefront: u = (p - P0) mod 4 is its ring slot, and
// U = (p - P0) mod 2 gives the exchange-buffer parities at compile time.
// Every row runs every stage: a row whose results no written column needs
// computes values that reach no output (rows beyond the window read the zero
// rows of the exchange arrays), and the stage code stays free of branches.
template <int RY, int U, int G>
__device__ __forceinline__ void tb2_plane(const StepArgs<float>& a, const Tb2Times& tt, const Tb2Col& c,
                                          const Tb2Bufs<RY>& b, Tb2Carry& s, bool valid, bool issue_next,
                                          float dt16, int u)
{
    using S = Tb2Smem<RY>;
    constexpr int NT = S::NT, NF = S::NF, XS = S::XS;
    constexpr bool GX = G & 1, GY = G & 2;
    const int SP = u, SQ = (u + 3) & 3, SR = (u + 2) & 3;   // slots of planes p, p-1, p-2
    constexpr int PP = U & 1, PQ = PP ^ 1;                        // exchange parities of planes p, p-1
    const int lane = c.lane, tid = c.tid;
    // (a window off the x faces, !GX, takes the edge lane's own value past
    // the window: lanes 0 and 31 are halo there, and what they compute
    // reaches no column the window writes)
    auto xp = [&](float v) {   // value of the +x neighbour (0 past the window)
        const float u = __shfl_down_sync(0xffffffffu, v, 1);
        return GX && lane == 31 ? 0.0f : u;
    };
    auto xm = [&](float v) {   // value of the -x neighbour
        const float u = __shfl_up_sync(0xffffffffu, v, 1);
        return GX && lane == 0 ? 0.0f : u;
    };
    // y neighbours from the padded exchange arrays (zero beyond the window)
    auto yp = [&](const float* q) { return q[S::XO + tid + 32]; };
    auto ym = [&](const float* q) { return q[S::XO + tid - 32]; };
    auto put = [&](float* q, float v) { q[S::XO + tid] = v; };
    const float cz = a.cz;

    cpa_wait2();   // this plane's fields and the last plane's psi (planes p + 1, p + 2 may still run)
    float* rp = b.ring + SP * NF * NT + tid;
    float* rq = b.ring + SQ * NF * NT + tid;
    float* rr = b.ring + SR * NF * NT + tid;
    // e^{i beta z} of plane p, used from the next plane on
    Cpx<float> zn{0.0f, 0.0f};
    if (c.ant) zn = static_cast<const Cpx<float>*>(a.zphr)[s.kp];

    // ---- stage A: H^{n+1/2} of plane q = p-1
    const float en0 = rp[0], en1 = rp[NT], en2 = rp[2 * NT];         // E^n(p)
    const float ex = s.e0[0], ey = s.e0[1], ez = s.e0[2];
    float hx = 0.0f, hy = 0.0f, hz = 0.0f, hsy = 0.0f;
    float nPEx = 0.0f, nPEy = 0.0f, ncz = 0.0f, nHsz = 0.0f, nhbx = 0.0f;
    {
        const float ox = rq[3 * NT], oy = rq[4 * NT], oz = rq[5 * NT];   // H^{n-1/2}(q)
        const float* EBq = b.EB + PQ * 2 * XS;
        const float ezj = yp(EBq), exj = yp(EBq + XS);
        const float ezi = xp(ez), eyi = xp(ey);
        const float dEz_y = ezj - ez, dEy_z = en1 - ey, dEx_z = en0 - ex;
        const float dEz_x = ezi - ez, dEy_x = eyi - ey, dEx_y = exj - ex;
        hx = ox - c.chy * dEz_y + cz * dEy_z;
        hy = oy - cz * dEx_z + c.chx * dEz_x;
        hz = oz - c.chx * dEy_x + c.chy * dEx_y;
        if (GX) {   // every lane (zero coefficients and psi off the x shells)
            const float p0 = psi_rn(c.bhx, rq[6 * NT], c.ahx, dEz_x);   // Hyx
            const float p1 = psi_rn(c.bhx, rq[7 * NT], c.ahx, dEy_x);   // Hzx
            hy += p0;
            hz -= p1;
            rq[6 * NT] = p0; rq[7 * NT] = p1;
        }
        if (GY && c.sy) {
            const float p0 = psi_rn(c.bhy, rq[8 * NT], c.ahy, dEz_y);   // Hxy
            const float p1 = psi_rn(c.bhy, rq[9 * NT], c.ahy, dEx_y);   // Hzy
            hx -= p0;
            hz += p1;
            rq[8 * NT] = p0; rq[9 * NT] = p1;
        }
        if (c.anth) {   // the whole row: zero terms where a column has no point
            const Cpx<float> u = cmul(s.zq, tt.th0);
            hx += tb2_src(b, c, 3, u);
            hy += tb2_src(b, c, 4, u);
            hz += tb2_src(b, c, 5, u);
        }
        // centre sums of step n for plane q
        nPEx = ex + exj;
        nPEy = ey + eyi;
        ncz = (ez + ezi) + (ezj + xp(ezj));
        const float hsx = ox + hx;
        hsy = oy + hy;
        nHsz = oz + hz;
        nhbx = hsx + xp(hsx);
    }
    {
        float* EBp = b.EB + PP * 2 * XS;
        put(EBp, en2);
        put(EBp + XS, en0);
        put(b.HB, hx);
        put(b.HB + XS, hz);
        put(b.HB + 2 * XS, hsy);
    }
    __syncthreads();

    // ---- stage B: E^{n+1} of plane q
    float nex = 0.0f, ney = 0.0f, nez = 0.0f;
    {
        const float hyi = xm(hy), hzi = xm(hz);
        const float hxj = ym(b.HB), hzj = ym(b.HB + XS);
        const float dHz_y = hz - hzj, dHy_z = hy - s.h1p[1], dHx_z = hx - s.h1p[0];
        const float dHz_x = hz - hzi, dHy_x = hy - hyi, dHx_y = hx - hxj;
        nex = ex + c.cey * dHz_y - cz * dHy_z;
        ney = ey + cz * dHx_z - c.cex * dHz_x;
        nez = ez + c.cex * dHy_x - c.cey * dHx_y;
        if (GX) {   // every lane (zero coefficients and psi off the x shells)
            const float p0 = psi_rn(c.bex, rq[10 * NT], c.aex, dHz_x);   // Eyx
            const float p1 = psi_rn(c.bex, rq[11 * NT], c.aex, dHy_x);   // Ezx
            rq[10 * NT] = p0; rq[11 * NT] = p1;
            ney -= p0;
            nez += p1;
        }
        if (GY && c.sy) {
            const float p0 = psi_rn(c.bey, rq[12 * NT], c.aey, dHz_y);   // Exy
            const float p1 = psi_rn(c.bey, rq[13 * NT], c.aey, dHx_y);   // Ezy
            rq[12 * NT] = p0; rq[13 * NT] = p1;
            nex += p0;
            nez -= p1;
        }
        if (c.ante) {   // the whole row: zero terms where a column has no point
            const Cpx<float> u = cmul(s.zq, tt.te0);
            nex += tb2_src(b, c, 0, u);
            ney += tb2_src(b, c, 1, u);
            nez += tb2_src(b, c, 2, u);
        }
        if (GY && c.j == 0) { nex = 0.0f; nez = 0.0f; }   // PEC: tangential E
        if (GX && c.i == 0) { ney = 0.0f; nez = 0.0f; }
    }
    // fluence term of step n for plane r (sums of planes r and q)
    float nhby = 0.0f, tn_new = 0.0f;
    {
        nhby = hsy + yp(b.HB + 2 * XS);
        tn_new = tb2_flux(s.fPEx + nPEx, s.fPEy + nPEy, s.fcz, s.fhbx, s.fhby, s.fHsz + nHsz, dt16);
    }

    // ---- stage C: H^{n+3/2} of plane r = p-2
    float h2x = 0.0f, h2y = 0.0f, h2z = 0.0f, gsy = 0.0f;
    float mPEx = 0.0f, mPEy = 0.0f, mcz = 0.0f, mHsz = 0.0f, mhbx = 0.0f;
    {
        const float* E1Br = b.E1B + PP * 2 * XS;   // written one plane ago (parity of r = parity of p)
        const float fezj = yp(E1Br), fexj = yp(E1Br + XS);
        const float fezi = xp(s.e1p[2]), feyi = xp(s.e1p[1]);
        const float dEz_y = fezj - s.e1p[2], dEy_z = ney - s.e1p[1], dEx_z = nex - s.e1p[0];
        const float dEz_x = fezi - s.e1p[2], dEy_x = feyi - s.e1p[1], dEx_y = fexj - s.e1p[0];
        h2x = s.h1p[0] - c.chy * dEz_y + cz * dEy_z;
        h2y = s.h1p[1] - cz * dEx_z + c.chx * dEz_x;
        h2z = s.h1p[2] - c.chx * dEy_x + c.chy * dEx_y;
        if (GX) {   // every lane (zero coefficients and psi off the x shells)
            const float p0 = psi_rn(c.bhx, rr[6 * NT], c.ahx, dEz_x);
            const float p1 = psi_rn(c.bhx, rr[7 * NT], c.ahx, dEy_x);
            h2y += p0;
            h2z -= p1;
            if (valid && c.own && c.sx) {
                const int qo = s.kr * a.ny * (2 * a.npml) + c.colx;
                const uint64_t pol = tb2_store_policy();
                st_keep(a.phx_out[0] + qo, p0, pol); st_keep(a.phx_out[1] + qo, p1, pol);
            }
        }
        if (GY && c.sy) {
            const float p0 = psi_rn(c.bhy, rr[8 * NT], c.ahy, dEz_y);
            const float p1 = psi_rn(c.bhy, rr[9 * NT], c.ahy, dEx_y);
            h2x -= p0;
            h2z += p1;
            if (valid && c.own) {
                const int qo = s.kr * (2 * a.npml) * a.pitch + c.coly;
                const uint64_t pol = tb2_store_policy();
                st_keep(a.phy_out[0] + qo, p0, pol); st_keep(a.phy_out[1] + qo, p1, pol);
            }
        }
        if (c.anth) {   // the whole row: zero terms where a column has no point
            const Cpx<float> u = cmul(s.zr, tt.th1);
            h2x += tb2_src(b, c, 3, u);
            h2y += tb2_src(b, c, 4, u);
            h2z += tb2_src(b, c, 5, u);
        }
        // centre sums of step n+1 for plane r
        mPEx = s.e1p[0] + fexj;
        mPEy = s.e1p[1] + feyi;
        mcz = (s.e1p[2] + fezi) + (fezj + xp(fezj));
        const float gsx = s.h1p[0] + h2x;
        gsy = s.h1p[1] + h2y;
        mHsz = s.h1p[2] + h2z;
        mhbx = gsx + xp(gsx);
    }
    {
        float* E1Bq = b.E1B + PQ * 2 * XS;
        put(E1Bq, nez);
        put(E1Bq + XS, nex);
        put(b.H1B, h2x);
        put(b.H1B + XS, h2z);
        put(b.H1B + 2 * XS, gsy);
    }
    __syncthreads();

    // ---- stage D: E^{n+2} of plane r
    {
        const float hyi = xm(h2y), hzi = xm(h2z);
        const float hxj = ym(b.H1B), hzj = ym(b.H1B + XS);
        const float dHz_y = h2z - hzj, dHy_z = h2y - s.h2py, dHx_z = h2x - s.h2px;
        const float dHz_x = h2z - hzi, dHy_x = h2y - hyi, dHx_y = h2x - hxj;
        float fx = s.e1p[0] + c.cey * dHz_y - cz * dHy_z;
        float fy = s.e1p[1] + cz * dHx_z - c.cex * dHz_x;
        float fz = s.e1p[2] + c.cex * dHy_x - c.cey * dHx_y;
        if (GX) {   // every lane (zero coefficients and psi off the x shells)
            const float p0 = psi_rn(c.bex, rr[10 * NT], c.aex, dHz_x);
            const float p1 = psi_rn(c.bex, rr[11 * NT], c.aex, dHy_x);
            fy -= p0;
            fz += p1;
            if (valid && c.own && c.sx) {
                const int qo = s.kr * a.ny * (2 * a.npml) + c.colx;
                const uint64_t pol = tb2_store_policy();
                st_keep(a.pex_out[0] + qo, p0, pol); st_keep(a.pex_out[1] + qo, p1, pol);
            }
        }
        if (GY && c.sy) {
            const float p0 = psi_rn(c.bey, rr[12 * NT], c.aey, dHz_y);
            const float p1 = psi_rn(c.bey, rr[13 * NT], c.aey, dHx_y);
            fx += p0;
            fz -= p1;
            if (valid && c.own) {
                const int qo = s.kr * (2 * a.npml) * a.pitch + c.coly;
                const uint64_t pol = tb2_store_policy();
                st_keep(a.pey_out[0] + qo, p0, pol); st_keep(a.pey_out[1] + qo, p1, pol);
            }
        }
        if (c.ante) {   // the whole row: zero terms where a column has no point
            const Cpx<float> u = cmul(s.zr, tt.te1);
            fx += tb2_src(b, c, 0, u);
            fy += tb2_src(b, c, 1, u);
            fz += tb2_src(b, c, 2, u);
        }
        if (GY && c.j == 0) { fx = 0.0f; fz = 0.0f; }
        if (GX && c.i == 0) { fy = 0.0f; fz = 0.0f; }
        if (valid && c.own) {
            const int g = s.kr * (a.pitch * a.ny) + c.col;
            const uint64_t pol = tb2_store_policy();
            st_keep(a.eout[0] + g, fx, pol); st_keep(a.eout[1] + g, fy, pol); st_keep(a.eout[2] + g, fz, pol);
            st_keep(a.hout[0] + g, h2x, pol); st_keep(a.hout[1] + g, h2y, pol); st_keep(a.hout[2] + g, h2z, pol);
        }
    }
    // fluence of plane p-3: the step-n term from the last plane, then step n+1
    float mhby = 0.0f;
    {   // every lane computes it (no divergent branch); the fluence cells store it
        mhby = gsy + yp(b.H1B + 2 * XS);
        const float t1 = tb2_flux(s.gPEx + mPEx, s.gPEy + mPEy, s.gcz, s.ghbx, s.ghby, s.gHsz + mHsz, dt16);
        float2 acc = b.fring[SP * NT + tid];   // zero-filled off the fluence cells
        acc = FluAcc<float>::add(acc, s.tn);
        acc = FluAcc<float>::add(acc, t1);
        if (valid && c.fown)
            st_keep(static_cast<float2*>(a.fluence) + s.k3 * (a.pitch * a.ny) + c.col, acc, tb2_store_policy());
    }

    // ---- carry to the next plane
    s.e0[0] = en0; s.e0[1] = en1; s.e0[2] = en2;
    s.h1p[0] = hx; s.h1p[1] = hy; s.h1p[2] = hz;
    s.e1p[0] = nex; s.e1p[1] = ney; s.e1p[2] = nez;
    s.h2px = h2x; s.h2py = h2y;
    s.fPEx = nPEx; s.fPEy = nPEy; s.fcz = ncz; s.fhbx = nhbx; s.fhby = nhby; s.fHsz = nHsz;
    s.gPEx = mPEx; s.gPEy = mPEy; s.gcz = mcz; s.ghbx = mhbx; s.ghby = mhby; s.gHsz = mHsz;
    s.tn = tn_new;
    s.zr = s.zq; s.zq = zn;
    // refill: the fields of plane p + 3 (fluence plane p) into the slot of
    // plane p - 1, whose fields were last read at this plane's stage A, and
    // the psi of plane p + 2 into the slot of plane p - 2, whose psi were last
    // read at this plane's stage D
    if (issue_next) tb2_issue<RY, G>(a, c, b, SQ, s.ki, s.kp, SR, next_plane(next_plane(s.kp, a.nz), a.nz));
    else cpa_commit();
    s.k3 = s.kr; s.kr = s.kq; s.kq = s.kp;
    s.kp = next_plane(s.kp, a.nz);
    s.ki = next_plane(s.ki, a.nz);
}

// One window, planes [kb, ke) of its E^{n+2} / H^{n+3/2} output (fluence
// planes [kb-1, ke-1), modulo nz).
template <int RY, int G>
__device__ __forceinline__ void tb2_window(const StepArgs<float>& a, const Tb2Times& tt, const Tb2Plan& tw,
                                           int window, int kb, int ke, const Tb2Bufs<RY>& b)
{
    constexpr int NT = Tb2Smem<RY>::NT;
    Tb2Col c;
    c.lane = threadIdx.x; c.row = threadIdx.y; c.tid = c.row * 32 + c.lane;
    const int nx = a.nx, ny = a.ny, nz = a.nz, npml = a.npml, w2 = 2 * npml;
    const int wx = window % tw.T, wy = window / tw.T;
    const int L0 = kTb2Sx * wx, M0 = (RY - 4) * wy;
    c.i = L0 + c.lane; c.j = M0 + c.row;
    c.indom = c.i < nx && c.j < ny;
    // E^{n+2} / H^{n+3/2} columns this window writes, and its fluence columns
    const int xa = wx == 0 ? 0 : L0 + 2, xb = wx == tw.T - 1 ? nx : L0 + kTb2Wx - 2;
    const int ya = wy == 0 ? 0 : M0 + 2, yb = wy == tw.U - 1 ? ny : M0 + RY - 2;
    c.own = c.i >= xa && c.i < xb && c.j >= ya && c.j < yb;
    const int fxa = wx == 0 ? 0 : xa - 1, fxb = wx == tw.T - 1 ? nx : xb - 1;
    const int fya = wy == 0 ? 0 : ya - 1, fyb = wy == tw.U - 1 ? ny : yb - 1;
    c.fown = a.fluence != nullptr && c.i >= fxa && c.i < fxb && c.j >= fya && c.j < fyb;
    c.sx = c.indom && npml > 0 && (c.i < npml || c.i >= nx - npml);
    c.sy = c.indom && npml > 0 && (c.j < npml || c.j >= ny - npml);
    const int ii = c.sx ? (c.i < npml ? c.i : c.i - nx + w2) : 0;
    const int jj = c.sy ? (c.j < npml ? c.j : c.j - ny + w2) : 0;
    c.col = c.indom ? c.j * a.pitch + c.i : 0;
    c.colx = c.sx ? c.j * w2 + ii : 0;
    c.coly = c.sy ? jj * a.pitch + c.i : 0;
    // coefficients of a column past the box are zero: its values stay zero
    c.chx = c.indom ? a.chx[c.i] : 0.0f; c.chy = c.indom ? a.chy[c.j] : 0.0f;
    c.cex = c.indom ? a.cex[c.i] : 0.0f; c.cey = c.indom ? a.cey[c.j] : 0.0f;
    c.bhx = c.sx ? a.bhx[ii] : 0.0f; c.ahx = c.sx ? a.ahx[ii] : 0.0f;
    c.bex = c.sx ? a.bex[ii] : 0.0f; c.aex = c.sx ? a.aex[ii] : 0.0f;
    c.bhy = c.sy ? a.bhy[jj] : 0.0f; c.ahy = c.sy ? a.ahy[jj] : 0.0f;
    c.bey = c.sy ? a.bey[jj] : 0.0f; c.aey = c.sy ? a.aey[jj] : 0.0f;
    c.mk = (c.indom && a.smask) ? (a.smask[c.j * nx + c.i] & 0x3f) : uint8_t(0);
    c.ant = __syncthreads_or(c.mk != 0) != 0;
    c.anth = __any_sync(0xffffffffu, (c.mk & 0x38) != 0);
    c.ante = __any_sync(0xffffffffu, (c.mk & 0x07) != 0);
    if (c.ant) {   // every column of the window, zeros where it has no point of a component
        const Cpx<float>* coef = static_cast<const Cpx<float>*>(a.scoefr);
        for (int q = 0; q < 6; ++q) {
            const Cpx<float> v = (c.mk >> q) & 1 ? coef[q * nx * ny + c.j * nx + c.i] : Cpx<float>{0.0f, 0.0f};
            b.SC[q * NT + c.tid] = make_float2(v.x, v.y);
        }
    }

    const float dt16 = float(a.dt16);
    const int P0 = kb - 2, P1 = ke + 1;   // planes streamed: kb-2 .. ke+1
    Tb2Carry s;
    for (int q = 0; q < 3; ++q) { s.e0[q] = 0.0f; s.h1p[q] = 0.0f; s.e1p[q] = 0.0f; }
    s.h2px = s.h2py = 0.0f;
    s.fPEx = s.fPEy = s.fcz = s.fhbx = s.fhby = s.fHsz = 0.0f;
    s.gPEx = s.gPEy = s.gcz = s.ghbx = s.ghby = s.gHsz = 0.0f;
    s.tn = 0.0f;
    s.zq = s.zr = Cpx<float>{0.0f, 0.0f};
    s.kp = (P0 % nz + nz) % nz;
    s.kq = s.kp == 0 ? nz - 1 : s.kp - 1;
    s.kr = s.kq == 0 ? nz - 1 : s.kq - 1;
    s.k3 = s.kr == 0 ? nz - 1 : s.kr - 1;
    // prologue: the fields of planes P0, P0 + 1, P0 + 2 into slots 0, 1, 2
    // (their fluence planes P0 - 3, P0 - 2, P0 - 1), the psi of planes P0 - 1,
    // P0, P0 + 1 into slots 3, 0, 1
    const int k1 = next_plane(s.kp, nz), k2 = next_plane(k1, nz);
    tb2_issue<RY, G>(a, c, b, 0, s.kp, s.k3, 3, s.kq);
    tb2_issue<RY, G>(a, c, b, 1, k1, s.kr, 0, s.kp);
    tb2_issue<RY, G>(a, c, b, 2, k2, s.kq, 1, k1);
    s.ki = next_plane(k2, nz);
    // the ring's four slots: plane p uses slot u = (p - P0) mod 4
    int p = P0;
    int u = 0;
    for (;;) {
        tb2_plane<RY, 0, G>(a, tt, c, b, s, p >= kb + 2, p + 3 <= P1, dt16, u);
        u = (u + 1) & 3;
        if (++p > P1) break;
        tb2_plane<RY, 1, G>(a, tt, c, b, s, p >= kb + 2, p + 3 <= P1, dt16, u);
        u = (u + 1) & 3;
        if (++p > P1) break;
    }
    cpa_wait0();
}

template <int RY>
__device__ __forceinline__ void tb2_run(const StepArgs<float>& a, const Tb2Times& tt, const Tb2Plan& tw)
{
    using S = Tb2Smem<RY>;
    constexpr int NT = S::NT, R = S::R, NF = S::NF;
    extern __shared__ __align__(16) unsigned char tb2_smem[];
    Tb2Bufs<RY> b;
    b.fring = reinterpret_cast<float2*>(tb2_smem);
    b.ring = reinterpret_cast<float*>(b.fring + R * NT);
    constexpr int XS = S::XS;
    b.EB = b.ring + R * NF * NT;
    b.HB = b.EB + 4 * XS;
    b.E1B = b.HB + 3 * XS;
    b.H1B = b.E1B + 4 * XS;
    b.SC = reinterpret_cast<float2*>(b.H1B + 3 * XS + 32);
    // the NX + 1 zero rows of the exchange arrays (never written again; the
    // first window's barrier orders these stores before any read)
    for (int q = threadIdx.y * 32 + threadIdx.x; q < (S::NX + 1) * 32; q += NT)
        b.EB[(q / 32) * XS + q % 32] = 0.0f;
    const long long t0 = tw.prof ? clock64() : 0;
    long long w = tw.start[blockIdx.x];
    const long long wend = tw.start[blockIdx.x + 1];
    while (w < wend) {
        const int window = tb2_window_at(tw, int(w / a.nz)), kb = int(w % a.nz);
        const long long left = wend - w;
        const int ke = left < (long long)(a.nz - kb) ? kb + int(left) : a.nz;
        // a window off the box faces and the CPML shells runs without the
        // checks of walls, psi and columns past the box (G = 0; the x and y
        // checks are separate flags, but instantiating them apart measured no
        // faster)
        const int wx = window % tw.T, wy = window / tw.T;
        const int L0 = kTb2Sx * wx, M0 = (RY - 4) * wy;
        const bool gen = wx == 0 || wx == tw.T - 1 || wy == 0 || wy == tw.U - 1 ||
                         (a.npml > 0 && (L0 < a.npml || L0 + kTb2Wx > a.nx - a.npml || M0 < a.npml ||
                                         M0 + RY > a.ny - a.npml));
        if (gen) tb2_window<RY, 3>(a, tt, tw, window, kb, ke, b);
        else tb2_window<RY, 0>(a, tt, tw, window, kb, ke, b);
        w += ke - kb;
        __syncthreads();   // the exchange buffers are reused by the next window
    }
    if (tw.prof && threadIdx.x == 0 && threadIdx.y == 0)
        tw.prof[blockIdx.x] += static_cast<unsigned long long>(clock64() - t0);
}

// Steps n and n+1 with their source time factors as a parameter.
template <int RY>
__global__ void __launch_bounds__(32 * RY, 1)
yee_tb2(const StepArgs<float> a, const Tb2Times tt, const __grid_constant__ Tb2Plan tw)
{
    tb2_run<RY>(a, tt, tw);
}

// The same with the time factors of the two steps read from a device table
// (times[i0] for step n, times[i1] for step n+1): the batched graph replays
// these launches with the table refreshed before each replay.
template <int RY>
__global__ void __launch_bounds__(32 * RY, 1)
yee_tb2_t(const StepArgs<float> a, const StepTime<float>* __restrict__ times, int i0, int i1,
          const __grid_constant__ Tb2Plan tw)
{
    Tb2Times tt;
    tt.th0 = times[i0].th; tt.te0 = times[i0].te;
    tt.th1 = times[i1].th; tt.te1 = times[i1].te;
    tb2_run<RY>(a, tt, tw);
}

}  // namespace fdtd
