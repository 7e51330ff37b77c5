// mlb_passes.cu -- the two force passes of one time step on sm_103a:
// pass 1: hard core (Eq. potmeanforce), velocity exchange (Eqs. gammaab,
// viscousforce) at u, the friction matrix and the half-step predictor;
// pass 2: velocity exchange at u* -> acceleration.  Shared-memory tiled
// (shell reach 1, 2) and global-memory variants.
#include "mlb_internal.h"
#include "mlb_device.cuh"

namespace {

// ------------------------------------------------------------------ pass 1
// Solve (I + G/2) x = b for symmetric G = (xx, yy, zz, xy, xz, yz).
__device__ __forceinline__ void solve_sym3(const float G[6], const float b[3], float x[3])
{
    float a00 = 1.f + 0.5f * G[0], a11 = 1.f + 0.5f * G[1], a22 = 1.f + 0.5f * G[2];
    float a01 = 0.5f * G[3], a02 = 0.5f * G[4], a12 = 0.5f * G[5];
    float c00 = a11 * a22 - a12 * a12;
    float c01 = a02 * a12 - a01 * a22;
    float c02 = a01 * a12 - a02 * a11;
    float c11 = a00 * a22 - a02 * a02;
    float c12 = a01 * a02 - a00 * a12;
    float c22 = a00 * a11 - a01 * a01;
    float inv = 1.f / (a00 * c00 + a01 * c01 + a02 * c02);
    x[0] = (c00 * b[0] + c01 * b[1] + c02 * b[2]) * inv;
    x[1] = (c01 * b[0] + c11 * b[1] + c12 * b[2]) * inv;
    x[2] = (c02 * b[0] + c12 * b[1] + c22 * b[2]) * inv;
}

// neighbour data of species b at r + sign*d (zero density beyond a wall)
struct Nb {
    float Dn, n, u0, u1, u2;
    long long q;
};

template <bool INTERIOR>
__device__ __forceinline__ Nb fetch_nb(const mlbi_params &p, const Loc &L, const float4 &e0, const float4 &e1,
                                       int sign, const float4 *__restrict__ fld, float nref, float dn0, float n0)
{
    Nb o;
    o.q = INTERIOR ? L.r + sign * (long long)__float_as_int(e1.x) : nbr(p, L, e0, e1, sign);
    if (INTERIOR || o.q >= 0) {
        const float4 v = fld[o.q];
        o.Dn = v.x - dn0; o.n = nref + v.x; o.u0 = v.y; o.u1 = v.z; o.u2 = v.w;
    } else {
        o.Dn = -n0; o.n = 0.f; o.u0 = 0.f; o.u1 = 0.f; o.u2 = 0.f;
    }
    return o;
}

// Shell sums of pass 1 for every species a over neighbour species b:
//   hard core  -hc_ab sum_{+-d} s (g(r)+g(r+d))/2 n^b(r+d)                   (Eq. potmeanforce)
//   exchange   vx_ab sum_{+-d} s s.[(g(r)+g(r+d))/2 n^b(r+d) (u^b(r+d) - u^a)]  (Eqs. gammaab, viscousforce)
//   friction   Gamma^a = vx_ab sum_{+-d} s s^T (g(r)+g(r+d))/2 n^b(r+d)
template <int S, bool INTERIOR>
__device__ __forceinline__ void pass1_shells(const mlbi_params &p, const Loc &L, const Centre<S> &c,
                                             const float *dgc, const float4 *__restrict__ mom,
                                             const float *__restrict__ dg, const mlbi_entry *__restrict__ tab,
                                             float (&hc)[S][3], float (&fv)[S][3], float (&G)[S][6])
{
    const long long N = p.N;
#pragma unroll
    for (int b = 0; b < S; ++b) {
        const float n0 = c.n[b], dn0 = c.dn[b];
        const int k0 = p.ushell_start[b], k1 = k0 + p.ushell_count[b];
        const float4 *fb = mom + b * N;
#pragma unroll 2
        for (int k = k0; k < k1; ++k) {
            const float4 e0 = __ldg(&tab[2 * k]);
            const float4 e1 = __ldg(&tab[2 * k + 1]);
            const int mask = __float_as_int(e1.y);
            const Nb P = fetch_nb<INTERIOR>(p, L, e0, e1, 1, fb, p.nref[b], dn0, n0);
            const Nb M = fetch_nb<INTERIOR>(p, L, e0, e1, -1, fb, p.nref[b], dn0, n0);
            const float sx = e0.x, sy = e0.y, sz = e0.z;
#pragma unroll
            for (int a = 0; a < S; ++a) {
                if (!(mask & (1 << a))) continue;
                const int q = pair_of(a, b, S);
                const mlbi_pair &pr = p.pair[q];
                const float *dgq = dg + q * N;
                const float Dgp = (INTERIOR || P.q >= 0) ? dgq[P.q] - dgc[q] : 0.f;
                const float Dgm = (INTERIOR || M.q >= 0) ? dgq[M.q] - dgc[q] : 0.f;
                const float g0 = pr.g_ref + dgc[q];
                // (g(r)+g(r+d))/2 n(r+d) - (g(r)+g(r-d))/2 n(r-d), expanded about site r
                const float t = -pr.hc_pre * (g0 * (P.Dn - M.Dn) + 0.5f * n0 * (Dgp - Dgm) +
                                              0.5f * (Dgp * P.Dn - Dgm * M.Dn));
                hc[a][0] += sx * t; hc[a][1] += sy * t; hc[a][2] += sz * t;
                const float gp = pr.vx_pre * (g0 + 0.5f * Dgp), gm = pr.vx_pre * (g0 + 0.5f * Dgm);
                const float wn = gp * P.n + gm * M.n;
                float w0, w1, w2;
                if (p.drag_only) {
                    w0 = wn * (c.u[b][0] - c.u[a][0]);
                    w1 = wn * (c.u[b][1] - c.u[a][1]);
                    w2 = wn * (c.u[b][2] - c.u[a][2]);
                } else {
                    const float hp = gp * P.n, hm = gm * M.n;
                    w0 = hp * (P.u0 - c.u[a][0]) + hm * (M.u0 - c.u[a][0]);
                    w1 = hp * (P.u1 - c.u[a][1]) + hm * (M.u1 - c.u[a][1]);
                    w2 = hp * (P.u2 - c.u[a][2]) + hm * (M.u2 - c.u[a][2]);
                }
                const float sd = sx * w0 + sy * w1 + sz * w2;
                fv[a][0] += sx * sd; fv[a][1] += sy * sd; fv[a][2] += sz * sd;
                G[a][0] += wn * sx * sx; G[a][1] += wn * sy * sy; G[a][2] += wn * sz * sz;
                G[a][3] += wn * sx * sy; G[a][4] += wn * sx * sz; G[a][5] += wn * sy * sz;
            }
        }
    }
}

// attraction sum_{+d} K_ab(d) (n^b(r+d) - n^b(r-d))  (G term of Eq. potmeanforce, RPA)
template <int S, bool INTERIOR>
__device__ __forceinline__ void pass1_attraction(const mlbi_params &p, const Loc &L,
                                                 const float4 *__restrict__ mom,
                                                 const mlbi_entry *__restrict__ tab, float (&at)[S][3])
{
    const long long N = p.N;
#pragma unroll
    for (int a = 0; a < S; ++a) {
#pragma unroll
        for (int b = 0; b < S; ++b) {
            const mlbi_pair &pr = p.pair[pair_of(a, b, S)];
            const float *nb = reinterpret_cast<const float *>(mom + b * N);
            float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll 4
            for (int k = pr.attr_start; k < pr.attr_start + pr.attr_count; ++k) {
                const float4 e0 = __ldg(&tab[2 * k]);
                const float4 e1 = __ldg(&tab[2 * k + 1]);
                float vp, vm;
                if (INTERIOR) {
                    const long long o = __float_as_int(e1.x);
                    vp = nb[4 * (L.r + o)];
                    vm = nb[4 * (L.r - o)];
                } else {
                    const long long ip = nbr(p, L, e0, e1, 1), im = nbr(p, L, e0, e1, -1);
                    // beyond a wall n = 0, i.e. n - n_ref = -n_ref
                    vp = ip >= 0 ? nb[4 * ip] : -p.nref[b];
                    vm = im >= 0 ? nb[4 * im] : -p.nref[b];
                }
                const float d = vp - vm;        // deviations cancel n_ref exactly inside the fluid
                s0 += e0.x * d; s1 += e0.y * d; s2 += e0.z * d;
            }
            at[a][0] += s0; at[a][1] += s1; at[a][2] += s2;
        }
    }
}

// pass 1: the shell and attraction sums at u, then du from
// (I + Gamma/2) du = (rest + exchange)/2 (one Jacobi sweep of u* = u + a(u*)/2
// with partner velocities held at u) and the inputs of pass 2.
template <int S>
__global__ void __launch_bounds__(kBX * kBY) k_pass1(const mlbi_params p, const float4 *__restrict__ mom,
                                                     const float *__restrict__ dg,
                                                     const mlbi_entry *__restrict__ tab,
                                                     const float4 *__restrict__ fext,
                                                     const float4 *__restrict__ attr, float4 *__restrict__ frest,
                                                     float4 *__restrict__ pst, float4 *__restrict__ du_out)
{
    constexpr int NP = S * (S + 1) / 2;
    Loc L;
    if (!locate(p, L)) return;
    const long long N = p.N, r = L.r;
    Centre<S> c;
    load_centre<S>(p, mom, r, c);
    float dgc[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) dgc[q] = dg[q * N + r];
    float hc[S][3], fv[S][3], G[S][6], at[S][3];
#pragma unroll
    for (int a = 0; a < S; ++a) {
#pragma unroll
        for (int k = 0; k < 3; ++k) { hc[a][k] = 0.f; fv[a][k] = 0.f; at[a][k] = 0.f; }
#pragma unroll
        for (int k = 0; k < 6; ++k) G[a][k] = 0.f;
    }
    if (L.interior) pass1_shells<S, true>(p, L, c, dgc, mom, dg, tab, hc, fv, G);
    else pass1_shells<S, false>(p, L, c, dgc, mom, dg, tab, hc, fv, G);
    if (p.attr_r) {
#pragma unroll
        for (int a = 0; a < S; ++a) {
            const float4 v = attr[a * N + r];
            at[a][0] = v.x; at[a][1] = v.y; at[a][2] = v.z;
        }
    } else if (p.has_attraction) {
        if (L.interior) pass1_attraction<S, true>(p, L, mom, tab, at);
        else pass1_attraction<S, false>(p, L, mom, tab, at);
    }
#pragma unroll
    for (int a = 0; a < S; ++a) {
        const float4 fe = p.has_fext ? fext[a * N + r] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float fr[3] = {hc[a][0] + at[a][0] + fe.x, hc[a][1] + at[a][1] + fe.y, hc[a][2] + at[a][2] + fe.z};
        float d[3] = {0.f, 0.f, 0.f};
        if (p.semi_implicit) {
            const float rhs[3] = {0.5f * (fr[0] + fv[a][0]), 0.5f * (fr[1] + fv[a][1]), 0.5f * (fr[2] + fv[a][2])};
            solve_sym3(G[a], rhs, d);
        }
        // pass 2 evaluates the exchange with the centre velocity u^a; -Gamma du completes it to u*
        const float gd0 = G[a][0] * d[0] + G[a][3] * d[1] + G[a][4] * d[2];
        const float gd1 = G[a][3] * d[0] + G[a][1] * d[1] + G[a][5] * d[2];
        const float gd2 = G[a][4] * d[0] + G[a][5] * d[1] + G[a][2] * d[2];
        if (p.drag_only) {
            frest[a * N + r] = make_float4(fr[0], fr[1], fr[2], 0.f);
            du_out[a * N + r] = make_float4(d[0], d[1], d[2], 0.f);
        } else {
            frest[a * N + r] = make_float4(fr[0] - gd0, fr[1] - gd1, fr[2] - gd2, 0.f);
        }
        pst[a * N + r] = make_float4(c.dn[a], c.u[a][0] + d[0], c.u[a][1] + d[1], c.u[a][2] + d[2]);
    }
}

// ------------------------------------------------------------------ pass 2: acceleration
// a^a = frest^a + vx_ab sum_{+-d} s s.[(g(r)+g(r+d))/2 n^b(r+d) (u*^b(r+d) - u^a)]
// with u* = u + du from pass 1 (drag only: partner velocity u*^b(r)).
template <int S, bool INTERIOR>
__device__ __forceinline__ void pass2_shells(const mlbi_params &p, const Loc &L, const Centre<S> &c,
                                             const float *dgc, const float (&us)[S][3],
                                             const float4 *__restrict__ pst, const float *__restrict__ dg,
                                             const mlbi_entry *__restrict__ tab, float (&acc)[S][3])
{
    const long long N = p.N;
#pragma unroll
    for (int b = 0; b < S; ++b) {
        const int k0 = p.ushell_start[b], k1 = k0 + p.ushell_count[b];
        const float4 *fb = pst + b * N;
#pragma unroll 2
        for (int k = k0; k < k1; ++k) {
            const float4 e0 = __ldg(&tab[2 * k]);
            const float4 e1 = __ldg(&tab[2 * k + 1]);
            const int mask = __float_as_int(e1.y);
            const Nb P = fetch_nb<INTERIOR>(p, L, e0, e1, 1, fb, p.nref[b], 0.f, 0.f);
            const Nb M = fetch_nb<INTERIOR>(p, L, e0, e1, -1, fb, p.nref[b], 0.f, 0.f);
            const float sx = e0.x, sy = e0.y, sz = e0.z;
#pragma unroll
            for (int a = 0; a < S; ++a) {
                if (!(mask & (1 << a))) continue;
                const int q = pair_of(a, b, S);
                const mlbi_pair &pr = p.pair[q];
                const float *dgq = dg + q * N;
                const float Dgp = (INTERIOR || P.q >= 0) ? dgq[P.q] - dgc[q] : 0.f;
                const float Dgm = (INTERIOR || M.q >= 0) ? dgq[M.q] - dgc[q] : 0.f;
                const float g0 = pr.g_ref + dgc[q];
                const float gp = pr.vx_pre * (g0 + 0.5f * Dgp), gm = pr.vx_pre * (g0 + 0.5f * Dgm);
                const float wn = gp * P.n + gm * M.n;
                float w0, w1, w2;
                if (p.drag_only) {
                    w0 = wn * (us[b][0] - us[a][0]);
                    w1 = wn * (us[b][1] - us[a][1]);
                    w2 = wn * (us[b][2] - us[a][2]);
                } else {
                    const float hp = gp * P.n, hm = gm * M.n;
                    w0 = hp * (P.u0 - c.u[a][0]) + hm * (M.u0 - c.u[a][0]);
                    w1 = hp * (P.u1 - c.u[a][1]) + hm * (M.u1 - c.u[a][1]);
                    w2 = hp * (P.u2 - c.u[a][2]) + hm * (M.u2 - c.u[a][2]);
                }
                const float sd = sx * w0 + sy * w1 + sz * w2;
                acc[a][0] += sx * sd; acc[a][1] += sy * sd; acc[a][2] += sz * sd;   // masses are 1
            }
        }
    }
}

template <int S>
__global__ void __launch_bounds__(kBX * kBY) k_pass2(const mlbi_params p, const float4 *__restrict__ mom,
                                                     const float *__restrict__ dg,
                                                     const mlbi_entry *__restrict__ tab,
                                                     const float4 *__restrict__ frest,
                                                     const float4 *__restrict__ pst,
                                                     const float4 *__restrict__ du, float4 *__restrict__ acc_f,
                                                     double *__restrict__ acc_out)
{
    constexpr int NP = S * (S + 1) / 2;
    Loc L;
    if (!locate(p, L)) return;
    const long long N = p.N, r = L.r;
    Centre<S> c;
    load_centre<S>(p, mom, r, c);
    float dgc[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) dgc[q] = dg[q * N + r];
    float us[S][3];                 // partner velocities at r (drag only)
#pragma unroll
    for (int a = 0; a < S; ++a) {
        if (p.drag_only) {
            const float4 v = du[a * N + r];
            us[a][0] = c.u[a][0] + v.x; us[a][1] = c.u[a][1] + v.y; us[a][2] = c.u[a][2] + v.z;
        } else {
            us[a][0] = 0.f; us[a][1] = 0.f; us[a][2] = 0.f;
        }
    }
    float acc[S][3];
#pragma unroll
    for (int a = 0; a < S; ++a) {
        const float4 fr = frest[a * N + r];
        acc[a][0] = fr.x; acc[a][1] = fr.y; acc[a][2] = fr.z;
    }
    if (L.interior) pass2_shells<S, true>(p, L, c, dgc, us, pst, dg, tab, acc);
    else pass2_shells<S, false>(p, L, c, dgc, us, pst, dg, tab, acc);
#pragma unroll
    for (int a = 0; a < S; ++a) {
        if (acc_out) {
#pragma unroll
            for (int q = 0; q < 3; ++q) acc_out[(a * 3 + q) * N + r] = (double)acc[a][q];
        } else {
            acc_f[a * N + r] = make_float4(acc[a][0], acc[a][1], acc[a][2], 0.f);
        }
    }
}

// The 13 canonical half offsets of the 3x3x3 cube (first non-zero of (dz, dy, dx)
// positive); with reach 1 every contact shell is a subset of them.
__device__ constexpr int KX[13] = {1, -1, 0, 1, -1, 0, 1, -1, 0, 1, -1, 0, 1};
__device__ constexpr int KY[13] = {0, 1, 1, 1, -1, -1, -1, 0, 0, 0, 1, 1, 1};
__device__ constexpr int KZ[13] = {0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 1, 1, 1};

__device__ __forceinline__ float cube_inv_len(int k)
{
    const int q = KX[k] * KX[k] + KY[k] * KY[k] + KZ[k] * KZ[k];
    return q == 1 ? 1.0f : (q == 2 ? 0.70710678118654752f : 0.57735026918962576f);
}

// ------------------------------------------------------------------ shared-memory tiles (z marching)
// A block of 32 x 4 threads owns a 32 x 4 column of sites and marches up z
// through `zchunk` planes.  The stencil field of every species (float4: the
// moments in pass 1, (n - n_ref, p*) in pass 2) and the contact-value
// deviations of every pair are staged in shared memory as a ring of planes
// of (32 + 2R) x (4 + 2R) sites: 2R + 1 planes in use and one more being
// filled by cp.async while the current plane is computed.  Every shell
// neighbour is then read from shared memory.
template <int S, int R>
struct Tile {
    static constexpr int TX = kBX, TY = kBY;
    static constexpr int TXH = TX + 2 * R, TYH = TY + 2 * R, PLANE = TXH * TYH;
    static constexpr int NSLOT = 2 * R + 2;
    static constexpr int NP = S * (S + 1) / 2;
    static constexpr size_t bytes = (size_t)NSLOT * PLANE * (S * sizeof(float4) + NP * sizeof(float));
};

// Stage plane gz of the tile with corner (x0 - R, y0 - R) into ring slot `slot`.
// Sites beyond a wall get n = 0 (n - n_ref = -n_ref), zero momentum and g = g_ref.
template <int S, int R>
__device__ __forceinline__ void stage_plane(const mlbi_params &p, int x0, int y0, int gz, int slot,
                                            const float4 *__restrict__ fld, const float *__restrict__ dg,
                                            float4 *sf, float *sg)
{
    using T = Tile<S, R>;
    const long long N = p.N;
    const int tid = threadIdx.y * kBX + threadIdx.x;
    const int z = wrap_or_out(gz, p.nz, p.wall_axis == 2);
    for (int idx = tid; idx < T::PLANE; idx += kBX * kBY) {
        const int hx = idx % T::TXH, hy = idx / T::TXH;
        const int x = wrap_or_out(x0 - R + hx, p.nx, p.wall_axis == 0);
        const int y = wrap_or_out(y0 - R + hy, p.ny, p.wall_axis == 1);
        float4 *df = sf + (size_t)slot * S * T::PLANE + idx;
        float *dgs = sg + (size_t)slot * T::NP * T::PLANE + idx;
        if (x < 0 || y < 0 || z < 0) {
#pragma unroll
            for (int b = 0; b < S; ++b) df[b * T::PLANE] = make_float4(-p.nref[b], 0.f, 0.f, 0.f);
#pragma unroll
            for (int q = 0; q < T::NP; ++q) dgs[q * T::PLANE] = 0.f;
        } else {
            const long long g = x + (long long)p.nx * (y + (long long)p.ny * z);
#pragma unroll
            for (int b = 0; b < S; ++b) cp_async16(df + b * T::PLANE, fld + b * N + g);
#pragma unroll
            for (int q = 0; q < T::NP; ++q) cp_async4(dgs + q * T::PLANE, dg + q * N + g);
        }
    }
}


// Shell sums of pass 1 from the tile (same sums as pass1_shells).
template <int S, int R>
__device__ __forceinline__ void pass1_tile_shells(const mlbi_params &p, const mlbi_entry *__restrict__ tab,
                                                  const float4 *sf, const float *sg, int kz,
                                                  int cidx, const Centre<S> &c, const float *dgc,
                                                  float (&hc)[S][3], float (&fv)[S][3], float (&G)[S][6])
{
    using T = Tile<S, R>;
#pragma unroll
    for (int b = 0; b < S; ++b) {
        const float n0 = c.n[b], dn0 = c.dn[b], nr = p.nref[b];
        const int k0 = p.ushell_start[b], k1 = k0 + p.ushell_count[b];
#pragma unroll 2
        for (int k = k0; k < k1; ++k) {
            const float4 e0 = __ldg(&tab[2 * k]);
            const float4 e1 = __ldg(&tab[2 * k + 1]);
            const int mask = __float_as_int(e1.y), off = __float_as_int(e1.z), dz = __float_as_int(e1.w);
            const int sp = ring(kz + dz, T::NSLOT), sm = ring(kz - dz, T::NSLOT);   // ring slots of the +-d planes
            const float4 vp = sf[sp * S * T::PLANE + b * T::PLANE + cidx + off];
            const float4 vm = sf[sm * S * T::PLANE + b * T::PLANE + cidx - off];
            const float Dnp = vp.x - dn0, np = nr + vp.x, Dnm = vm.x - dn0, nm = nr + vm.x;
            const float sx = e0.x, sy = e0.y, sz = e0.z;
#pragma unroll
            for (int a = 0; a < S; ++a) {
                if (!(mask & (1 << a))) continue;
                const int q = pair_of(a, b, S);
                const mlbi_pair &pr = p.pair[q];
                const float Dgp = sg[sp * T::NP * T::PLANE + q * T::PLANE + cidx + off] - dgc[q];
                const float Dgm = sg[sm * T::NP * T::PLANE + q * T::PLANE + cidx - off] - dgc[q];
                const float g0 = pr.g_ref + dgc[q];
                const float t = -pr.hc_pre * (g0 * (Dnp - Dnm) + 0.5f * n0 * (Dgp - Dgm) +
                                              0.5f * (Dgp * Dnp - Dgm * Dnm));
                hc[a][0] += sx * t; hc[a][1] += sy * t; hc[a][2] += sz * t;
                const float gp = pr.vx_pre * (g0 + 0.5f * Dgp), gm = pr.vx_pre * (g0 + 0.5f * Dgm);
                const float wn = gp * np + gm * nm;
                float w0, w1, w2;
                if (p.drag_only) {
                    w0 = wn * (c.u[b][0] - c.u[a][0]);
                    w1 = wn * (c.u[b][1] - c.u[a][1]);
                    w2 = wn * (c.u[b][2] - c.u[a][2]);
                } else {
                    const float hp = gp * np, hm = gm * nm;
                    w0 = hp * (vp.y - c.u[a][0]) + hm * (vm.y - c.u[a][0]);
                    w1 = hp * (vp.z - c.u[a][1]) + hm * (vm.z - c.u[a][1]);
                    w2 = hp * (vp.w - c.u[a][2]) + hm * (vm.w - c.u[a][2]);
                }
                const float sd = sx * w0 + sy * w1 + sz * w2;
                fv[a][0] += sx * sd; fv[a][1] += sy * sd; fv[a][2] += sz * sd;
                G[a][0] += wn * sx * sx; G[a][1] += wn * sy * sy; G[a][2] += wn * sz * sz;
                G[a][3] += wn * sx * sy; G[a][4] += wn * sx * sz; G[a][5] += wn * sy * sz;
            }
        }
    }
}

// Pass-1 shell sums for reach 1: the 13 half offsets of the 3x3x3 cube are
// compile-time constants, so the unit vectors are immediates and their zero
// components drop out; cube_mask[pair] selects the offsets of each shell.
template <int S>
__device__ __forceinline__ void pass1_cube_shells(const mlbi_params &p, const float4 *sf, const float *sg, int kz,
                                                  int cidx, const Centre<S> &c, const float *dgc,
                                                  float (&hc)[S][3], float (&fv)[S][3], float (&G)[S][6])
{
    using T = Tile<S, 1>;
    // ring slots of the planes z - 1, z, z + 1 as element offsets (32-bit)
    const int s4[3] = {ring(kz - 1, T::NSLOT) * S * T::PLANE + cidx, ring(kz, T::NSLOT) * S * T::PLANE + cidx,
                       ring(kz + 1, T::NSLOT) * S * T::PLANE + cidx};
    const int s1[3] = {ring(kz - 1, T::NSLOT) * T::NP * T::PLANE + cidx, ring(kz, T::NSLOT) * T::NP * T::PLANE + cidx,
                       ring(kz + 1, T::NSLOT) * T::NP * T::PLANE + cidx};
#pragma unroll
    for (int b = 0; b < S; ++b) {
        const float n0 = c.n[b], dn0 = c.dn[b], nr = p.nref[b];
        int any = 0;
#pragma unroll
        for (int a = 0; a < S; ++a) any |= p.cube_mask[pair_of(a, b, S)];
#pragma unroll
        for (int k = 0; k < 13; ++k) {
            if (!((any >> k) & 1)) continue;
            const int off = KX[k] + T::TXH * KY[k];
            const float4 vp = sf[s4[1 + KZ[k]] + b * T::PLANE + off];
            const float4 vm = sf[s4[1 - KZ[k]] + b * T::PLANE - off];
            const float dDn = vp.x - vm.x, np = nr + vp.x, nm = nr + vm.x;
            const float il = cube_inv_len(k);
            const float sx = KX[k] * il, sy = KY[k] * il, sz = KZ[k] * il;
            const bool hx = KX[k] != 0, hy = KY[k] != 0, hz = KZ[k] != 0;
            // s . u at +-d, shared by every species a
            float sjp = 0.f, sjm = 0.f;
            if (hx) { sjp += sx * vp.y; sjm += sx * vm.y; }
            if (hy) { sjp += sy * vp.z; sjm += sy * vm.z; }
            if (hz) { sjp += sz * vp.w; sjm += sz * vm.w; }
#pragma unroll
            for (int a = 0; a < S; ++a) {
                const int q = pair_of(a, b, S);
                if (!((p.cube_mask[q] >> k) & 1)) continue;
                const mlbi_pair &pr = p.pair[q];
                const float Dgp = sg[s1[1 + KZ[k]] + q * T::PLANE + off] - dgc[q];
                const float Dgm = sg[s1[1 - KZ[k]] + q * T::PLANE - off] - dgc[q];
                const float g0 = pr.g_ref + dgc[q];
                // (g(r)+g(r+d))/2 n(r+d) - (g(r)+g(r-d))/2 n(r-d) = g0 (n+ - n-) + (n+ Dg+ - n- Dg-)/2
                const float t = -pr.hc_pre * (g0 * dDn + 0.5f * (np * Dgp - nm * Dgm));
                if (hx) hc[a][0] += sx * t;
                if (hy) hc[a][1] += sy * t;
                if (hz) hc[a][2] += sz * t;
                const float gp = pr.vx_pre * (g0 + 0.5f * Dgp), gm = pr.vx_pre * (g0 + 0.5f * Dgm);
                const float wn = gp * np + gm * nm;
                float su = 0.f;                    // s . u^a (drag only: s . (u^b - u^a))
                if (p.drag_only) {
                    if (hx) su += sx * (c.u[a][0] - c.u[b][0]);
                    if (hy) su += sy * (c.u[a][1] - c.u[b][1]);
                    if (hz) su += sz * (c.u[a][2] - c.u[b][2]);
                } else {
                    if (hx) su += sx * c.u[a][0];
                    if (hy) su += sy * c.u[a][1];
                    if (hz) su += sz * c.u[a][2];
                }
                const float sd = p.drag_only ? -wn * su : gp * np * (sjp - su) + gm * nm * (sjm - su);
                if (hx) fv[a][0] += sx * sd;
                if (hy) fv[a][1] += sy * sd;
                if (hz) fv[a][2] += sz * sd;
                if (hx) G[a][0] += wn * (sx * sx);
                if (hy) G[a][1] += wn * (sy * sy);
                if (hz) G[a][2] += wn * (sz * sz);
                if (hx && hy) G[a][3] += wn * (sx * sy);
                if (hx && hz) G[a][4] += wn * (sx * sz);
                if (hy && hz) G[a][5] += wn * (sy * sz);
            }
        }
    }
}

// Pass-2 exchange sums for reach 1 (the cube specialisation of the table loop).
template <int S>
__device__ __forceinline__ void pass2_cube_shells(const mlbi_params &p, const float4 *sf, const float *sg, int kz,
                                                  int cidx, const Centre<S> &c, const float *dgc,
                                                  const float (&us)[S][3], float (&acc)[S][3])
{
    using T = Tile<S, 1>;
    const int s4[3] = {ring(kz - 1, T::NSLOT) * S * T::PLANE + cidx, ring(kz, T::NSLOT) * S * T::PLANE + cidx,
                       ring(kz + 1, T::NSLOT) * S * T::PLANE + cidx};
    const int s1[3] = {ring(kz - 1, T::NSLOT) * T::NP * T::PLANE + cidx, ring(kz, T::NSLOT) * T::NP * T::PLANE + cidx,
                       ring(kz + 1, T::NSLOT) * T::NP * T::PLANE + cidx};
#pragma unroll
    for (int b = 0; b < S; ++b) {
        const float nr = p.nref[b];
        int any = 0;
#pragma unroll
        for (int a = 0; a < S; ++a) any |= p.cube_mask[pair_of(a, b, S)];
#pragma unroll
        for (int k = 0; k < 13; ++k) {
            if (!((any >> k) & 1)) continue;
            const int off = KX[k] + T::TXH * KY[k];
            const float4 vp = sf[s4[1 + KZ[k]] + b * T::PLANE + off];
            const float4 vm = sf[s4[1 - KZ[k]] + b * T::PLANE - off];
            const float np = nr + vp.x, nm = nr + vm.x;
            const float il = cube_inv_len(k);
            const float sx = KX[k] * il, sy = KY[k] * il, sz = KZ[k] * il;
            const bool hx = KX[k] != 0, hy = KY[k] != 0, hz = KZ[k] != 0;
            float sjp = 0.f, sjm = 0.f;              // s . u* at +-d, shared by every species a
            if (hx) { sjp += sx * vp.y; sjm += sx * vm.y; }
            if (hy) { sjp += sy * vp.z; sjm += sy * vm.z; }
            if (hz) { sjp += sz * vp.w; sjm += sz * vm.w; }
#pragma unroll
            for (int a = 0; a < S; ++a) {
                const int q = pair_of(a, b, S);
                if (!((p.cube_mask[q] >> k) & 1)) continue;
                const mlbi_pair &pr = p.pair[q];
                const float Dgp = sg[s1[1 + KZ[k]] + q * T::PLANE + off] - dgc[q];
                const float Dgm = sg[s1[1 - KZ[k]] + q * T::PLANE - off] - dgc[q];
                const float g0 = pr.g_ref + dgc[q];
                const float gp = pr.vx_pre * (g0 + 0.5f * Dgp), gm = pr.vx_pre * (g0 + 0.5f * Dgm);
                const float wn = gp * np + gm * nm;
                float su = 0.f;                    // s . u^a (drag only: s . (u*^a - u*^b))
                if (p.drag_only) {
                    if (hx) su += sx * (us[a][0] - us[b][0]);
                    if (hy) su += sy * (us[a][1] - us[b][1]);
                    if (hz) su += sz * (us[a][2] - us[b][2]);
                } else {
                    if (hx) su += sx * c.u[a][0];
                    if (hy) su += sy * c.u[a][1];
                    if (hz) su += sz * c.u[a][2];
                }
                const float sd = p.drag_only ? -wn * su : gp * np * (sjp - su) + gm * nm * (sjm - su);
                if (hx) acc[a][0] += sx * sd;     // masses are 1
                if (hy) acc[a][1] += sy * sd;
                if (hz) acc[a][2] += sz * sd;
            }
        }
    }
}

template <int S>
__device__ __forceinline__ void centre_from(const mlbi_params &p, const float4 (&v)[S], Centre<S> &c)
{
#pragma unroll
    for (int a = 0; a < S; ++a) {
        c.dn[a] = v[a].x;
        c.n[a] = p.nref[a] + v[a].x;
        c.u[a][0] = v[a].y; c.u[a][1] = v[a].z; c.u[a][2] = v[a].w;
    }
}

// finish pass 1 at one site: predictor and outputs (shared by both pass-1 kernels)
template <int S>
__device__ __forceinline__ void pass1_finish(const mlbi_params &p, long long r, const Centre<S> &c,
                                             const float (&hc)[S][3], const float (&fv)[S][3],
                                             const float (&G)[S][6], const float (&at)[S][3],
                                             const float4 *__restrict__ fext, float4 *__restrict__ frest,
                                             float4 *__restrict__ pst, float4 *__restrict__ du_out)
{
    const long long N = p.N;
#pragma unroll
    for (int a = 0; a < S; ++a) {
        const float4 fe = p.has_fext ? fext[a * N + r] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float fr[3] = {hc[a][0] + at[a][0] + fe.x, hc[a][1] + at[a][1] + fe.y, hc[a][2] + at[a][2] + fe.z};
        float d[3] = {0.f, 0.f, 0.f};
        if (p.semi_implicit) {
            // one Jacobi sweep of u* = u + a(u*)/2 with partner velocities held at u
            const float rhs[3] = {0.5f * (fr[0] + fv[a][0]), 0.5f * (fr[1] + fv[a][1]), 0.5f * (fr[2] + fv[a][2])};
            solve_sym3(G[a], rhs, d);
        }
        // pass 2 evaluates the exchange with the centre velocity u^a; -Gamma du completes it to u*
        const float gd0 = G[a][0] * d[0] + G[a][3] * d[1] + G[a][4] * d[2];
        const float gd1 = G[a][3] * d[0] + G[a][1] * d[1] + G[a][5] * d[2];
        const float gd2 = G[a][4] * d[0] + G[a][5] * d[1] + G[a][2] * d[2];
        if (p.drag_only) {
            frest[a * N + r] = make_float4(fr[0], fr[1], fr[2], 0.f);
            du_out[a * N + r] = make_float4(d[0], d[1], d[2], 0.f);
        } else {
            frest[a * N + r] = make_float4(fr[0] - gd0, fr[1] - gd1, fr[2] - gd2, 0.f);
        }
        pst[a * N + r] = make_float4(c.dn[a], c.u[a][0] + d[0], c.u[a][1] + d[1], c.u[a][2] + d[2]);
    }
}

template <int S, int R>
__global__ void __launch_bounds__(kBX * kBY, 4) k_pass1_tiled(const mlbi_params p, const float4 *__restrict__ mom,
                                                              const float *__restrict__ dg,
                                                              const mlbi_entry *__restrict__ tab,
                                                              const float4 *__restrict__ fext,
                                                              const float4 *__restrict__ attr,
                                                              float4 *__restrict__ frest, float4 *__restrict__ pst,
                                                              float4 *__restrict__ du_out)
{
    using T = Tile<S, R>;
    extern __shared__ float4 smem[];
    float4 *sf = smem;                                                      // [NSLOT][S][PLANE]
    float *sg = reinterpret_cast<float *>(smem + (size_t)T::NSLOT * S * T::PLANE);   // [NSLOT][NP][PLANE]
    const int x0 = blockIdx.x * kBX, y0 = blockIdx.y * kBY, z0 = blockIdx.z * p.zchunk;
    const int z1 = min(z0 + p.zchunk, p.nz);
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const bool active = x < p.nx && y < p.ny;
    const int cidx = (threadIdx.y + R) * T::TXH + threadIdx.x + R;
    for (int k = 0; k < 2 * R + 1; ++k) stage_plane<S, R>(p, x0, y0, z0 - R + k, ring(k, T::NSLOT), mom, dg, sf, sg);
    cp_async_commit();
    for (int z = z0; z < z1; ++z) {
        cp_async_wait_all();
        __syncthreads();
        const int kz = z - z0 + R;                      // ring position of plane z
        if (z + 1 < z1) {
            stage_plane<S, R>(p, x0, y0, z + R + 1, ring(kz + R + 1, T::NSLOT), mom, dg, sf, sg);
            cp_async_commit();
        }
        if (!active) continue;
        const int cs = ring(kz, T::NSLOT);
        float4 cv[S];
#pragma unroll
        for (int a = 0; a < S; ++a) cv[a] = sf[cs * S * T::PLANE + a * T::PLANE + cidx];
        Centre<S> c;
        centre_from<S>(p, cv, c);
        float dgc[T::NP];
#pragma unroll
        for (int q = 0; q < T::NP; ++q) dgc[q] = sg[cs * T::NP * T::PLANE + q * T::PLANE + cidx];
        float hc[S][3], fv[S][3], G[S][6], at[S][3];
#pragma unroll
        for (int a = 0; a < S; ++a) {
#pragma unroll
            for (int k = 0; k < 3; ++k) { hc[a][k] = 0.f; fv[a][k] = 0.f; at[a][k] = 0.f; }
#pragma unroll
            for (int k = 0; k < 6; ++k) G[a][k] = 0.f;
        }
        if constexpr (R == 1) pass1_cube_shells<S>(p, sf, sg, kz, cidx, c, dgc, hc, fv, G);
        else pass1_tile_shells<S, R>(p, tab, sf, sg, kz, cidx, c, dgc, hc, fv, G);
        const long long r = x + (long long)p.nx * (y + (long long)p.ny * z);
        if (p.attr_r) {
#pragma unroll
            for (int a = 0; a < S; ++a) {
                const float4 v = attr[a * p.N + r];
                at[a][0] = v.x; at[a][1] = v.y; at[a][2] = v.z;
            }
        } else if (p.has_attraction) {
            Loc L;
            L.x = x; L.y = y; L.z = z; L.r = r;
            const int Rr = p.reach;
            L.interior = x >= Rr && x < p.nx - Rr && y >= Rr && y < p.ny - Rr && z >= Rr && z < p.nz - Rr;
            if (L.interior) pass1_attraction<S, true>(p, L, mom, tab, at);
            else pass1_attraction<S, false>(p, L, mom, tab, at);
        }
        pass1_finish<S>(p, r, c, hc, fv, G, at, fext, frest, pst, du_out);
    }
}

template <int S, int R>
__global__ void __launch_bounds__(kBX * kBY, 4) k_pass2_tiled(const mlbi_params p, const float4 *__restrict__ mom,
                                                              const float *__restrict__ dg,
                                                              const mlbi_entry *__restrict__ tab,
                                                              const float4 *__restrict__ frest,
                                                              const float4 *__restrict__ pst,
                                                              const float4 *__restrict__ du,
                                                              float4 *__restrict__ acc_f, double *__restrict__ acc_out)
{
    using T = Tile<S, R>;
    extern __shared__ float4 smem[];
    float4 *sf = smem;
    float *sg = reinterpret_cast<float *>(smem + (size_t)T::NSLOT * S * T::PLANE);
    const long long N = p.N;
    const int x0 = blockIdx.x * kBX, y0 = blockIdx.y * kBY, z0 = blockIdx.z * p.zchunk;
    const int z1 = min(z0 + p.zchunk, p.nz);
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const bool active = x < p.nx && y < p.ny;
    const int cidx = (threadIdx.y + R) * T::TXH + threadIdx.x + R;
    for (int k = 0; k < 2 * R + 1; ++k) stage_plane<S, R>(p, x0, y0, z0 - R + k, ring(k, T::NSLOT), pst, dg, sf, sg);
    cp_async_commit();
    for (int z = z0; z < z1; ++z) {
        cp_async_wait_all();
        __syncthreads();
        const int kz = z - z0 + R;
        if (z + 1 < z1) {
            stage_plane<S, R>(p, x0, y0, z + R + 1, ring(kz + R + 1, T::NSLOT), pst, dg, sf, sg);
            cp_async_commit();
        }
        if (!active) continue;
        const int cs = ring(kz, T::NSLOT);
        const long long r = x + (long long)p.nx * (y + (long long)p.ny * z);
        Centre<S> c;
        load_centre<S>(p, mom, r, c);
        float dgc[T::NP];
#pragma unroll
        for (int q = 0; q < T::NP; ++q) dgc[q] = sg[cs * T::NP * T::PLANE + q * T::PLANE + cidx];
        float us[S][3];
#pragma unroll
        for (int a = 0; a < S; ++a) {
            if (p.drag_only) {
                const float4 v = du[a * N + r];
                us[a][0] = c.u[a][0] + v.x; us[a][1] = c.u[a][1] + v.y; us[a][2] = c.u[a][2] + v.z;
            } else {
                us[a][0] = 0.f; us[a][1] = 0.f; us[a][2] = 0.f;
            }
        }
        float acc[S][3];
#pragma unroll
        for (int a = 0; a < S; ++a) {
            const float4 fr = frest[a * N + r];
            acc[a][0] = fr.x; acc[a][1] = fr.y; acc[a][2] = fr.z;
        }
        if constexpr (R == 1) {
            pass2_cube_shells<S>(p, sf, sg, kz, cidx, c, dgc, us, acc);
        } else {
#pragma unroll
        for (int b = 0; b < S; ++b) {
            const float nr = p.nref[b];
            const int k0 = p.ushell_start[b], k1 = k0 + p.ushell_count[b];
#pragma unroll 2
            for (int k = k0; k < k1; ++k) {
                const float4 e0 = __ldg(&tab[2 * k]);
                const float4 e1 = __ldg(&tab[2 * k + 1]);
                const int mask = __float_as_int(e1.y), off = __float_as_int(e1.z), dz = __float_as_int(e1.w);
                const int sp = ring(kz + dz, T::NSLOT), sm = ring(kz - dz, T::NSLOT);
                const float4 vp = sf[sp * S * T::PLANE + b * T::PLANE + cidx + off];
                const float4 vm = sf[sm * S * T::PLANE + b * T::PLANE + cidx - off];
                const float np = nr + vp.x, nm = nr + vm.x;
                const float sx = e0.x, sy = e0.y, sz = e0.z;
#pragma unroll
                for (int a = 0; a < S; ++a) {
                    if (!(mask & (1 << a))) continue;
                    const int q = pair_of(a, b, S);
                    const mlbi_pair &pr = p.pair[q];
                    const float Dgp = sg[sp * T::NP * T::PLANE + q * T::PLANE + cidx + off] - dgc[q];
                    const float Dgm = sg[sm * T::NP * T::PLANE + q * T::PLANE + cidx - off] - dgc[q];
                    const float g0 = pr.g_ref + dgc[q];
                    const float gp = pr.vx_pre * (g0 + 0.5f * Dgp), gm = pr.vx_pre * (g0 + 0.5f * Dgm);
                    const float wn = gp * np + gm * nm;
                    float w0, w1, w2;
                    if (p.drag_only) {
                        w0 = wn * (us[b][0] - us[a][0]);
                        w1 = wn * (us[b][1] - us[a][1]);
                        w2 = wn * (us[b][2] - us[a][2]);
                    } else {
                        const float hp = gp * np, hm = gm * nm;
                        w0 = hp * (vp.y - c.u[a][0]) + hm * (vm.y - c.u[a][0]);
                        w1 = hp * (vp.z - c.u[a][1]) + hm * (vm.z - c.u[a][1]);
                        w2 = hp * (vp.w - c.u[a][2]) + hm * (vm.w - c.u[a][2]);
                    }
                    const float sd = sx * w0 + sy * w1 + sz * w2;
                    acc[a][0] += sx * sd; acc[a][1] += sy * sd; acc[a][2] += sz * sd;   // masses are 1
                }
            }
        }
        }
#pragma unroll
        for (int a = 0; a < S; ++a) {
            if (acc_out) {
#pragma unroll
                for (int q = 0; q < 3; ++q) acc_out[(a * 3 + q) * N + r] = (double)acc[a][q];
            } else {
                acc_f[a * N + r] = make_float4(acc[a][0], acc[a][1], acc[a][2], 0.f);
            }
        }
    }
}

}  // namespace

#define MLBI_DISPATCH_S(...)                                                                       \
    switch (p.S) {                                                                                 \
    case 1: { constexpr int SS = 1; __VA_ARGS__; } break;                                          \
    case 2: { constexpr int SS = 2; __VA_ARGS__; } break;                                          \
    case 3: { constexpr int SS = 3; __VA_ARGS__; } break;                                          \
    case 4: { constexpr int SS = 4; __VA_ARGS__; } break;                                          \
    default: return cudaErrorInvalidValue;                                                         \
    }

template <int S, int R>
cudaError_t launch_pass1_tiled(const mlbi_params &p, const mlbi_buffers &b, cudaStream_t s)
{
    using T = Tile<S, R>;
    auto k = k_pass1_tiled<S, R>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::bytes);
    if (e != cudaSuccess) return e;
    const dim3 g((unsigned)((p.nx + kBX - 1) / kBX), (unsigned)((p.ny + kBY - 1) / kBY),
                 (unsigned)((p.nz + p.zchunk - 1) / p.zchunk));
    k<<<g, dim3(kBX, kBY), T::bytes, s>>>(p, b.mom, b.dg, b.table, b.fext, b.attr, b.frest, b.pst, b.du);
    return cudaGetLastError();
}

template <int S, int R>
cudaError_t launch_pass2_tiled(const mlbi_params &p, const mlbi_buffers &b, double *acc_out, cudaStream_t s)
{
    using T = Tile<S, R>;
    auto k = k_pass2_tiled<S, R>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::bytes);
    if (e != cudaSuccess) return e;
    const dim3 g((unsigned)((p.nx + kBX - 1) / kBX), (unsigned)((p.ny + kBY - 1) / kBY),
                 (unsigned)((p.nz + p.zchunk - 1) / p.zchunk));
    k<<<g, dim3(kBX, kBY), T::bytes, s>>>(p, b.mom, b.dg, b.table, b.frest, b.pst, b.du, b.acc, acc_out);
    return cudaGetLastError();
}

cudaError_t mlbi_launch_pass1(const mlbi_params &p, const mlbi_buffers &b, cudaStream_t s)
{
    if (p.tile_r == 1) { MLBI_DISPATCH_S(return launch_pass1_tiled<SS, 1>(p, b, s)); }
    if (p.tile_r == 2) { MLBI_DISPATCH_S(return launch_pass1_tiled<SS, 2>(p, b, s)); }
    const dim3 g = tiled_grid(p), t(kBX, kBY);
    MLBI_DISPATCH_S((k_pass1<SS><<<g, t, 0, s>>>(p, b.mom, b.dg, b.table, b.fext, b.attr, b.frest, b.pst, b.du)));
    return cudaGetLastError();
}

cudaError_t mlbi_launch_pass2(const mlbi_params &p, const mlbi_buffers &b, double *acc_out, cudaStream_t s)
{
    if (p.tile_r == 1) { MLBI_DISPATCH_S(return launch_pass2_tiled<SS, 1>(p, b, acc_out, s)); }
    if (p.tile_r == 2) { MLBI_DISPATCH_S(return launch_pass2_tiled<SS, 2>(p, b, acc_out, s)); }
    const dim3 g = tiled_grid(p), t(kBX, kBY);
    MLBI_DISPATCH_S((k_pass2<SS><<<g, t, 0, s>>>(p, b.mom, b.dg, b.table, b.frest, b.pst, b.du, b.acc, acc_out)));
    return cudaGetLastError();
}

