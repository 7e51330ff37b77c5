// mlb_api.cu -- the C ABI declared in include/mlb.h: context, validation,
// stencil tables, device memory and the launch sequence of one time step.
#include "mlb.h"
#include "mlb_internal.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

namespace {

constexpr int kTableCap = 16384;               // stencil entries per context (2 float4 each, 512 KiB)
constexpr double kPi = 3.14159265358979323846;
constexpr double kCs2 = 1.0 / 3.0;

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

struct mlb_ctx {
    mlb_lattice_desc desc{};
    mlbi_params p{};
    mlbi_buffers b{};
    mlbi_maps maps{};
    void *slab = nullptr;
    size_t slab_bytes = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int cur = 0;
    int64_t step = 0;
    bool species_set = false, fields_set = false;
    bool failed = false;
    std::string err;
    std::vector<double> sigma, mass, eps, lambda_c, nref;
    std::vector<mlbi_entry> table;
    int max_offset = 1;                         // largest stencil offset component
    // instrumentation: one event pair per recorded launch
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<int> ev_kind;                   // kernel kind of pair k
    size_t ev_used = 0;
    double prof_ms[16] = {0};
    int64_t prof_count[16] = {0};
    // Jacobi sweeps of the half step (mlb_set_predictor_sweeps); pst2 is the
    // second (n - n_ref, u*) buffer the sweeps alternate with, allocated on
    // the first request of more than one sweep; pst_final is where the last
    // sweep of the current step left u*
    int sweeps = 1;
    float4 *pst2 = nullptr;
    float4 *pst_final = nullptr;
    // tensor-core attraction (MLB_MEANFIELD_BF16): tables in their own device
    // allocation, rebuilt with the stencils
    mlbi_tc_tables tc{};
    void *tc_mem = nullptr;
    size_t tc_bytes = 0;
    // work decomposition chosen by mlb_autotune (0 / -1: the defaults)
    int tuned_zchunk = 0;
    int tuned_split = -1;
    // bumped whenever the kernels' parameters change (captured graphs go stale)
    uint64_t version = 0;
    // learned surrogate of the hard-core force (mlb_attach_surrogate)
    mlb_net *surr = nullptr;
    int surr_every = 0;
    double surr_bound = 0.0, surr_err = -1.0;
    bool surr_active = false;
    int64_t surr_rechecks = 0, surr_rejections = 0;
    double *surr_sums = nullptr;                // device [2]
};

namespace {

mlb_status fail(mlb_ctx *c, mlb_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
    if (s == MLB_ECUDA || s == MLB_ENUMERIC || s == MLB_ETIMEOUT) c->failed = true;
    return s;
}

mlb_status cuda_check(mlb_ctx *c, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return MLB_OK;
    return fail(c, MLB_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define MLB_GUARD(ctx)                                                                     \
    do {                                                                                   \
        if (!(ctx)) return MLB_EINVAL;                                                     \
        if ((ctx)->failed) return MLB_ESTATE;                                              \
    } while (0)

#define MLB_CUDA(ctx, call)                                                                \
    do {                                                                                   \
        mlb_status st_ = cuda_check((ctx), (call), #call);                                 \
        if (st_ != MLB_OK) return st_;                                                     \
    } while (0)

double bmcsl(double sa, double sb, double xi2, double xi3)
{
    double h = sa * sb / (sa + sb), o = 1.0 - xi3;
    return 1.0 / o + 3.0 * h * xi2 / (o * o) + 2.0 * h * h * xi2 * xi2 / (o * o * o);
}

// cuTensorMapEncodeTiled from the driver (through the runtime, so that the
// library links no driver library itself); NULL if unavailable
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)f;
    }
    return fn;
}

// TMA descriptors of the populations, moments and rest force for the fused
// pass-2 + collision kernel: boxes of one 32 x 4 tile row block of one z
// plane, all species (and all 19 populations) at once.  Rows of FP32
// populations must be 16-byte multiples, so nx % 4 == 0; otherwise (or if the
// driver lacks the call) maps.ok stays 0 and the kernel stages by cp.async.
void encode_maps(mlb_ctx *c)
{
    mlbi_maps &m = c->maps;
    m.ok = 0;
    const mlbi_params &p = c->p;
    EncodeTiledFn fn = encode_tiled();
    if (!fn || p.nx % 4 != 0) return;
    const cuuint64_t nx = p.nx, ny = p.ny, nz = p.nz, S = p.S;
    const cuuint32_t ones[5] = {1, 1, 1, 1, 1};
    {
        const cuuint64_t dims[4] = {nx, ny, nz, S * MLBI_Q};
        const cuuint64_t strides[3] = {nx * 4, nx * ny * 4, nx * ny * nz * 4};
        const cuuint32_t box[4] = {32, 4, 1, (cuuint32_t)(S * MLBI_Q)};
        for (int k = 0; k < 2; ++k)
            if (fn(&m.f[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, c->b.f[k], dims, strides, box, ones,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return;
    }
    {
        const cuuint64_t dims[5] = {4, nx, ny, nz, S};
        const cuuint64_t strides[4] = {16, nx * 16, nx * ny * 16, nx * ny * nz * 16};
        const cuuint32_t box[5] = {4, 32, 4, 1, (cuuint32_t)S};
        if (fn(&m.mom, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, c->b.mom, dims, strides, box, ones,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return;
        if (fn(&m.frest, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, c->b.frest, dims, strides, box, ones,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return;
    }
    m.ok = 1;
}

// canonical half of the +-d pairs: first non-zero of (dz, dy, dx) positive
bool canonical(int dx, int dy, int dz)
{
    return dz > 0 || (dz == 0 && (dy > 0 || (dy == 0 && dx > 0)));
}

// FP32 -> BF16 bits, round to nearest even (finite values)
uint16_t bf16_bits(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
float bf16_value(uint16_t b)
{
    const uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

void *ctx_alloc(mlb_ctx *c, size_t bytes)
{
    void *ptr = nullptr;
    if (c->desc.dev_alloc) return c->desc.dev_alloc(bytes, c->desc.alloc_user);
    return cudaMalloc(&ptr, bytes) == cudaSuccess ? ptr : nullptr;
}
void ctx_free(mlb_ctx *c, void *ptr)
{
    if (!ptr) return;
    if (c->desc.dev_free) c->desc.dev_free(ptr, c->desc.alloc_user);
    else cudaFree(ptr);
}

// Tables of the tensor-core attraction: the columns (dx, dy) of every pair's
// region sigma_ab <= |d| <= lambda_c sigma_ab, sorted by dy then dx, and per
// column the B operand of the band product along z, hi and lo BF16 parts of
// K_ab(dx, dy, z' - z)_c at row k = 32 b + z' - z0 + 8, column
// n = 16 (3 a + c) + z, in the K-major layout [k / 8][n][k % 8].
mlb_status build_tc_tables(mlb_ctx *c)
{
    const mlbi_params &p = c->p;
    const int S = p.S, R = p.attr_r;
    const int N = 48 * S, K = 32 * S, KC = K / 8;
    auto rc_of = [&](int a, int b) { return c->lambda_c[a * S + b] * 0.5 * (c->sigma[a] + c->sigma[b]); };
    auto kernel = [&](int a, int b, int dx, int dy, int dz, int comp) {
        const double e = c->eps[a * S + b], sab = 0.5 * (c->sigma[a] + c->sigma[b]), rc = rc_of(a, b);
        const double q = (double)(dx * dx + dy * dy + dz * dz);
        if (e == 0.0 || q == 0.0 || q < sab * sab || q > rc * rc) return 0.0;
        const double d[3] = {(double)dx, (double)dy, (double)dz};
        return 6.0 * e * std::pow(sab, 6.0) / (q * q * q * q) * d[comp];
    };
    std::vector<int2> cols;
    std::vector<int> row_start;
    for (int dy = -R; dy <= R; ++dy) {
        bool row = false;
        for (int dx = -R; dx <= R; ++dx) {
            bool any = false;
            for (int a = 0; a < S && !any; ++a)
                for (int b = 0; b < S && !any; ++b)
                    for (int dz = -R; dz <= R && !any; ++dz) any = kernel(a, b, dx, dy, dz, 0) != 0.0 ||
                                                                  kernel(a, b, dx, dy, dz, 1) != 0.0 ||
                                                                  kernel(a, b, dx, dy, dz, 2) != 0.0;
            if (!any) continue;
            if (!row) row_start.push_back((int)cols.size());
            row = true;
            cols.push_back(make_int2(dx, dy));
        }
    }
    row_start.push_back((int)cols.size());
    const size_t colb = mlbi_attraction_tc_column_bytes(S);
    std::vector<uint16_t> w(cols.size() * colb / 2, 0);
    for (size_t ci = 0; ci < cols.size(); ++ci) {
        uint16_t *hi = w.data() + ci * colb / 2, *lo = hi + (size_t)KC * N * 8;
        for (int k = 0; k < K; ++k)
            for (int n = 0; n < N; ++n) {
                const int b = k / 32, zz = k % 32, a = n / 48, comp = (n / 16) % 3, z = n % 16;
                const double v = kernel(a, b, cols[ci].x, cols[ci].y, zz - 8 - z, comp);
                const uint16_t h = bf16_bits((float)v);
                const uint16_t l = bf16_bits((float)(v - (double)bf16_value(h)));
                const size_t at = ((size_t)(k / 8) * N + n) * 8 + k % 8;
                hi[at] = h;
                lo[at] = l;
            }
    }
    int nxp = 0, nyp = 0;
    mlbi_attraction_tc_padded(p, &nxp, &nyp);
    const size_t qb = align256(sizeof(uint16_t) * (size_t)S * nxp * nyp * p.nz);
    const size_t need = align256(w.size() * 2) + align256(cols.size() * sizeof(int2)) +
                        align256(row_start.size() * sizeof(int)) + 2 * qb;
    if (need > c->tc_bytes) {
        ctx_free(c, c->tc_mem);
        c->tc_mem = ctx_alloc(c, need);
        c->tc_bytes = c->tc_mem ? need : 0;
        if (!c->tc_mem) return fail(c, MLB_ENOMEM, "tensor-core attraction tables (%zu bytes)", need);
    }
    char *m = (char *)c->tc_mem;
    c->tc.weights = m; m += align256(w.size() * 2);
    c->tc.cols = (int2 *)m; m += align256(cols.size() * sizeof(int2));
    c->tc.row_start = (int *)m; m += align256(row_start.size() * sizeof(int));
    c->tc.qhi = m; m += qb;
    c->tc.qlo = m;
    c->tc.ncols = (int)cols.size();
    c->tc.nrows = (int)row_start.size() - 1;
    c->tc.pass3 = (c->desc.flags & MLB_MEANFIELD_BF16_1PASS) ? 0 : 1;
    // tensor maps of the padded copies: dims (z, b, xp, yp), box (8 planes, 1, 144 sites, 1)
    MLB_CUDA(c, cudaMemcpyAsync(c->tc.weights, w.data(), w.size() * 2, cudaMemcpyHostToDevice, c->stream));
    MLB_CUDA(c, cudaMemcpyAsync(c->tc.cols, cols.data(), cols.size() * sizeof(int2), cudaMemcpyHostToDevice,
                                c->stream));
    MLB_CUDA(c, cudaMemcpyAsync(c->tc.row_start, row_start.data(), row_start.size() * sizeof(int),
                                cudaMemcpyHostToDevice, c->stream));
    MLB_CUDA(c, cudaStreamSynchronize(c->stream));
    return MLB_OK;
}

bool use_tc_attraction(const mlb_ctx *c)
{
    return (c->desc.flags & MLB_MEANFIELD_BF16) && c->p.attr_r && c->tc.ncols > 0;
}

// Rebuild every stencil table and the parameter block from species,
// interactions and reference densities.
mlb_status rebuild(mlb_ctx *c)
{
    const int S = c->desc.nspecies;
    const long long nx = c->desc.nx, nxy = (long long)c->desc.nx * c->desc.ny;
    mlbi_params &p = c->p;
    std::vector<mlbi_entry> tab;
    int maxoff = 1;
    bool lin_overflow = false;
    // reach of the union shells: the tiled kernels stage a halo of this width
    int shell_reach = 1;
    for (int a = 0; a < S; ++a)
        for (int b = 0; b < S; ++b) {
            const double sab = 0.5 * (c->sigma[a] + c->sigma[b]);
            shell_reach = std::max(shell_reach, (int)std::floor(std::sqrt(std::pow(sab + 0.5, 2) - 1e-9)));
        }
    const int tile_r = mlbi_tile_ty(S, shell_reach) ? shell_reach : 0;
    const int txh = 32 + 2 * tile_r;
    // reach of the attraction regions (column attraction kernel if <= 8)
    int attr_reach = 0;
    for (int a = 0; a < S; ++a)
        for (int b = 0; b < S; ++b)
            if (!c->eps.empty() && c->eps[a * S + b] != 0.0)
                attr_reach = std::max(attr_reach,
                                      (int)std::floor(c->lambda_c[a * S + b] * 0.5 * (c->sigma[a] + c->sigma[b]) + 1e-9));
    const int attr_r = (attr_reach >= 1 && attr_reach <= 8) ? attr_reach : 0;
    auto push = [&](int dx, int dy, int dz, double vx, double vy, double vz, int mask) {
        mlbi_entry e0, e1;
        e0.x = (float)vx; e0.y = (float)vy; e0.z = (float)vz;
        int packed = mlbi_pack(dx, dy, dz);
        std::memcpy(&e0.w, &packed, sizeof(int));
        long long lin = dx + nx * dy + nxy * dz;
        if (lin >= (1ll << 31) || lin <= -(1ll << 31)) lin_overflow = true;
        int lin32 = (int)lin, tileoff = dx + txh * dy, dzz = dz;
        std::memcpy(&e1.x, &lin32, sizeof(int));
        std::memcpy(&e1.y, &mask, sizeof(int));
        std::memcpy(&e1.z, &tileoff, sizeof(int));
        std::memcpy(&e1.w, &dzz, sizeof(int));
        tab.push_back(e0);
        tab.push_back(e1);
        maxoff = std::max(maxoff, std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz))));
    };
    auto count = [&]() { return (int)(tab.size() / 2); };
    // smoothing balls |d| <= kappa sigma_c (origin included)
    for (int g = 0; g < S; ++g) {
        double R = c->desc.kappa * c->sigma[g];
        int Ri = (int)std::floor(R) + 1;
        p.ball_start[g] = count();
        for (int dz = -Ri; dz <= Ri; ++dz)
            for (int dy = -Ri; dy <= Ri; ++dy)
                for (int dx = -Ri; dx <= Ri; ++dx)
                    if ((double)(dx * dx + dy * dy + dz * dz) <= R * R) push(dx, dy, dz, 0, 0, 0, 0);
        p.ball_count[g] = count() - p.ball_start[g];
        p.ball_inv[g] = 1.0f / (float)p.ball_count[g];
    }
    auto in_shell = [](double sab, int dx, int dy, int dz) {
        const double q = (double)(dx * dx + dy * dy + dz * dz), lo = sab - 0.5, hi = sab + 0.5;
        return q > 0.0 && q >= (lo > 0 ? lo * lo : 0.0) && q < hi * hi;
    };
    // pairs
    int np = 0;
    bool attraction = false;
    double xi2 = 0.0, xi3 = 0.0;
    for (int g = 0; g < S; ++g) {
        xi2 += kPi / 6.0 * c->sigma[g] * c->sigma[g] * c->nref[g];
        xi3 += kPi / 6.0 * c->sigma[g] * c->sigma[g] * c->sigma[g] * c->nref[g];
    }
    for (int a = 0; a < S; ++a)
        for (int b = a; b < S; ++b) {
            mlbi_pair &pr = p.pair[np];
            const double sab = 0.5 * (c->sigma[a] + c->sigma[b]);
            const int Ri = (int)std::ceil(sab + 0.5) + 1;
            pr.shell_start = count();
            for (int dz = -Ri; dz <= Ri; ++dz)
                for (int dy = -Ri; dy <= Ri; ++dy)
                    for (int dx = -Ri; dx <= Ri; ++dx) {
                        if (!canonical(dx, dy, dz) || !in_shell(sab, dx, dy, dz)) continue;
                        const double len = std::sqrt((double)(dx * dx + dy * dy + dz * dz));
                        push(dx, dy, dz, dx / len, dy / len, dz / len, 0);
                    }
            pr.shell_count = count() - pr.shell_start;
            const double wS = 4.0 * kPi / (2.0 * pr.shell_count);
            const double mu = c->mass[a] * c->mass[b] / (c->mass[a] + c->mass[b]);
            pr.hc_pre = (float)(c->desc.kT * sab * sab * wS);
            pr.vx_pre = (float)(2.0 * sab * sab * std::sqrt(2.0 * mu * c->desc.kT / kPi) * wS);
            pr.h = (float)(c->sigma[a] * c->sigma[b] / (c->sigma[a] + c->sigma[b]));
            pr.g_ref = (float)bmcsl(c->sigma[a], c->sigma[b], xi2, xi3);
            // attraction: K(d) = 6 eps sigma^6 d / |d|^8 on sigma <= |d| <= lambda_c sigma
            // (one entry per point of the half region, for reaches the column form does not serve)
            pr.attr_start = count();
            const double e = c->eps.empty() ? 0.0 : c->eps[a * S + b];
            if (e != 0.0) attraction = true;
            if (e != 0.0 && !attr_r) {
                const double rc = c->lambda_c[a * S + b] * sab;
                const int Rc = (int)std::ceil(rc) + 1;
                const double s6 = std::pow(sab, 6.0);
                for (int dz = -Rc; dz <= Rc; ++dz)
                    for (int dy = -Rc; dy <= Rc; ++dy)
                        for (int dx = -Rc; dx <= Rc; ++dx) {
                            const double q = (double)(dx * dx + dy * dy + dz * dz);
                            if (q == 0.0 || !canonical(dx, dy, dz)) continue;
                            if (q < sab * sab || q > rc * rc) continue;
                            const double k = 6.0 * e * s6 / (q * q * q * q);
                            push(dx, dy, dz, k * dx, k * dy, k * dz, 0);
                        }
            }
            pr.attr_count = count() - pr.attr_start;
            p.pair_index[a][b] = p.pair_index[b][a] = np;
            ++np;
        }
    // union half shells per neighbour species b, with a mask of the species a
    // whose pair shell (a, b) contains the offset
    for (int b = 0; b < S; ++b) {
        int R = 1;
        for (int a = 0; a < S; ++a) R = std::max(R, (int)std::ceil(0.5 * (c->sigma[a] + c->sigma[b]) + 0.5) + 1);
        p.ushell_start[b] = count();
        for (int dz = -R; dz <= R; ++dz)
            for (int dy = -R; dy <= R; ++dy)
                for (int dx = -R; dx <= R; ++dx) {
                    if (!canonical(dx, dy, dz)) continue;
                    int mask = 0;
                    for (int a = 0; a < S; ++a)
                        if (in_shell(0.5 * (c->sigma[a] + c->sigma[b]), dx, dy, dz)) mask |= 1 << a;
                    if (!mask) continue;
                    const double len = std::sqrt((double)(dx * dx + dy * dy + dz * dz));
                    push(dx, dy, dz, dx / len, dy / len, dz / len, mask);
                }
        p.ushell_count[b] = count() - p.ushell_start[b];
    }
    if (attraction) maxoff = std::max(maxoff, attr_reach);
    // column form of the attraction: the region sigma_ab <= |d| <= lambda_c sigma_ab
    // cut into columns (dx, dy) of the half plane; per column and pair the
    // profile k(dz) = 6 eps sigma^6 / |d|^8 (zero off the region) and dz k(dz)
    p.acol_start = p.acol_count = p.aw_start = 0;
    if (attraction && attr_r) {
        struct Col { int dx, dy, E; };
        std::vector<Col> cols;
        auto rc_of = [&](int a, int b) { return c->lambda_c[a * S + b] * 0.5 * (c->sigma[a] + c->sigma[b]); };
        for (int dy = 0; dy <= attr_r; ++dy)
            for (int dx = -attr_r; dx <= attr_r; ++dx) {
                if (dy == 0 && dx < 0) continue;                    // half plane, (0, 0) kept
                int E = -1;
                for (int a = 0; a < S; ++a)
                    for (int b = a; b < S; ++b) {
                        if (c->eps[a * S + b] == 0.0) continue;
                        const double rc = rc_of(a, b), sab = 0.5 * (c->sigma[a] + c->sigma[b]);
                        for (int dz = 0; dz <= attr_r; ++dz) {
                            const double q = (double)(dx * dx + dy * dy + dz * dz);
                            if (q > 0.0 && q >= sab * sab && q <= rc * rc) E = std::max(E, dz);
                        }
                    }
                if (E >= 0) cols.push_back({dx, dy, E});
            }
        p.acol_start = (int)tab.size();                            // float4 index
        for (const Col &k : cols) {
            mlbi_entry e;
            std::memcpy(&e.x, &k.dx, sizeof(int));
            std::memcpy(&e.y, &k.dy, sizeof(int));
            std::memcpy(&e.z, &k.E, sizeof(int));
            e.w = 0.f;
            tab.push_back(e);
        }
        p.acol_count = (int)cols.size();
        std::vector<float> w;                                       // (k, dz k) pairs
        for (const Col &k : cols)
            for (int a = 0; a < S; ++a)
                for (int b = a; b < S; ++b) {
                    const double e = c->eps[a * S + b], sab = 0.5 * (c->sigma[a] + c->sigma[b]);
                    const double rc = rc_of(a, b), s6 = std::pow(sab, 6.0);
                    for (int dz = 0; dz <= attr_r; ++dz) {
                        const double q = (double)(k.dx * k.dx + k.dy * k.dy + dz * dz);
                        const bool in = e != 0.0 && q > 0.0 && q >= sab * sab && q <= rc * rc;
                        const double kk = in ? 6.0 * e * s6 / (q * q * q * q) : 0.0;
                        // the (0, 0) column pairs with itself: its +-dz sum counts each point twice
                        const double half = (k.dx == 0 && k.dy == 0) ? 0.5 : 1.0;
                        w.push_back((float)kk);
                        w.push_back((float)(half * dz * kk));
                    }
                }
        while (w.size() % 4) w.push_back(0.f);
        p.aw_start = (int)tab.size();
        for (size_t i = 0; i < w.size(); i += 4) {
            mlbi_entry e;
            e.x = w[i]; e.y = w[i + 1]; e.z = w[i + 2]; e.w = w[i + 3];
            tab.push_back(e);
        }
    }
    if (lin_overflow) return fail(c, MLB_EINVAL, "stencil offsets exceed 32-bit linear offsets on this lattice");
    if (tab.size() > 2 * (size_t)kTableCap)
        return fail(c, MLB_EINVAL, "stencil tables need %d float4, capacity is %d (reduce sigma or lambda_c)",
                    (int)tab.size(), 2 * kTableCap);
    const int L[3] = {c->desc.nx, c->desc.ny, c->desc.nz};
    for (int ax = 0; ax < 3; ++ax)
        if (ax != c->desc.wall_axis && L[ax] <= maxoff)
            return fail(c, MLB_EINVAL,
                        "periodic extent %d along axis %d must exceed the largest stencil offset %d", L[ax], ax,
                        maxoff);
    p.npairs = np;
    p.has_attraction = attraction ? 1 : 0;
    p.local_g = 1;
    for (int g = 0; g < S; ++g)
        if (p.ball_count[g] != 1) p.local_g = 0;
    p.tile_r = tile_r;
    p.attr_r = attraction ? attr_r : 0;
    // planes per block of the stencil kernels unless tuned: 12 leaves shorter
    // last waves than 16 on large lattices (256^3: 0.5 % faster per step)
    p.zchunk = std::min(c->desc.nz, c->tuned_zchunk > 0 ? c->tuned_zchunk : 12);
    // the 13 canonical half offsets of the 3x3x3 cube, in the order the kernels use:
    // (1,0,0); (-1,1,0), (0,1,0), (1,1,0); then dz = 1 with dy = -1, 0, 1 and dx = -1, 0, 1
    {
        int cube[13][3], k = 0;
        cube[k][0] = 1; cube[k][1] = 0; cube[k][2] = 0; ++k;
        for (int dx = -1; dx <= 1; ++dx) { cube[k][0] = dx; cube[k][1] = 1; cube[k][2] = 0; ++k; }
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) { cube[k][0] = dx; cube[k][1] = dy; cube[k][2] = 1; ++k; }
        for (int a2 = 0; a2 < S; ++a2)
            for (int b2 = a2; b2 < S; ++b2) {
                const double sab = 0.5 * (c->sigma[a2] + c->sigma[b2]);
                int m = 0;
                for (int j = 0; j < 13; ++j)
                    if (in_shell(sab, cube[j][0], cube[j][1], cube[j][2])) m |= 1 << j;
                p.cube_mask[p.pair_index[a2][b2]] = m;
            }
    }
    p.reach = maxoff;
    p.xi2_ref = (float)xi2;
    p.xi3_ref = (float)xi3;
    for (int g = 0; g < S; ++g) {
        p.nref[g] = (float)c->nref[g];
        p.xi2_coef[g] = (float)(kPi / 6.0 * c->sigma[g] * c->sigma[g]);
        p.xi3_coef[g] = (float)(kPi / 6.0 * c->sigma[g] * c->sigma[g] * c->sigma[g]);
    }
    c->table = tab;
    c->max_offset = maxoff;
    MLB_CUDA(c, cudaMemcpyAsync((void *)c->b.table, tab.data(), tab.size() * sizeof(mlbi_entry),
                                cudaMemcpyHostToDevice, c->stream));
    MLB_CUDA(c, cudaStreamSynchronize(c->stream));
    c->tc.ncols = 0;
    if ((c->desc.flags & MLB_MEANFIELD_BF16) && p.has_attraction) {
        if (!mlbi_attraction_tc_supported(p))
            return fail(c, MLB_EINVAL,
                        "the BF16 tensor-core mean field needs 1 or 2 species, an attraction reach of 1..8, "
                        "nz a multiple of 8 and no walls normal to z");
        mlb_status st = build_tc_tables(c);
        if (st != MLB_OK) return st;
    }
    ++c->version;
    return MLB_OK;
}

// the status the fault-flag word fl stands for
mlb_status flags_status(mlb_ctx *c, unsigned int fl)
{
    if (fl & MLBI_FLAG_TIMEOUT) return fail(c, MLB_ETIMEOUT, "a bounded wait on a bulk tensor copy gave up");
    if (fl & MLBI_FLAG_NAN) return fail(c, MLB_ENUMERIC, "non-finite moments met (the state diverged)");
    if (fl & MLBI_FLAG_XI3) return fail(c, MLB_ENUMERIC, "packing fraction xi3 >= 1 met at some site");
    return MLB_OK;
}

mlb_status check_flags(mlb_ctx *c)
{
    unsigned int fl = 0;
    MLB_CUDA(c, cudaMemcpyAsync(&fl, c->b.flags, sizeof fl, cudaMemcpyDeviceToHost, c->stream));
    MLB_CUDA(c, cudaStreamSynchronize(c->stream));
    return flags_status(c, fl);
}

mlb_status require_ready(mlb_ctx *c)
{
    if (!c->species_set) return fail(c, MLB_ESTATE, "mlb_set_species has not been called");
    if (!c->fields_set) return fail(c, MLB_ESTATE, "no state: call mlb_set_fields or mlb_set_populations");
    return MLB_OK;
}

enum {
    K_MOMENTS = 0, K_GFIELD = 1, K_PASS1 = 2, K_PASS2 = 3, K_COLLIDE = 4, K_ATTRACTION = 5, K_PASS2_COLLIDE = 6,
    K_SURROGATE = 7, K_SWEEP = 8, K_NKINDS = 9
};
const char *const kKernelNames[K_NKINDS] = {"k_moments", "k_gfield", "k_pass1", "k_pass2", "k_collide",
                                            "k_attraction", "k_pass2_collide", "k_surrogate", "k_sweep"};

// event pair around one launch when profiling
struct Timed {
    mlb_ctx *c;
    size_t k = (size_t)-1;
    Timed(mlb_ctx *ctx, int kind) : c(ctx)
    {
        if (!c->profiling) return;
        if (c->ev_used * 2 + 2 > c->ev_pool.size()) {
            cudaEvent_t e0, e1;
            if (cudaEventCreate(&e0) != cudaSuccess) return;
            if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return; }
            c->ev_pool.push_back(e0);
            c->ev_pool.push_back(e1);
            c->ev_kind.push_back(kind);
        }
        k = c->ev_used++;
        c->ev_kind[k] = kind;
        cudaEventRecord(c->ev_pool[2 * k], c->stream);
    }
    ~Timed()
    {
        if (k != (size_t)-1) cudaEventRecord(c->ev_pool[2 * k + 1], c->stream);
    }
};

mlb_status forces_pass1(mlb_ctx *c, bool sums);

// Further Jacobi sweeps of the half step after pass 1 (pass 1 is the first):
// u* alternates between b.pst and pst2; pst_final marks the last one.
mlb_status sweeps(mlb_ctx *c)
{
    c->pst_final = c->b.pst;
    if (!c->p.semi_implicit) return MLB_OK;
    for (int k = 1; k < c->sweeps; ++k) {
        float4 *next = c->pst_final == c->b.pst ? c->pst2 : c->b.pst;
        Timed t(c, K_SWEEP);
        MLB_CUDA(c, mlbi_launch_sweep(c->p, c->b, c->pst_final, next, c->stream));
        c->pst_final = next;
    }
    return MLB_OK;
}

// The force passes of one step on the current populations; sums: the moment
// pass also leaves the FP64 conservation sums of the state in b.sums.
mlb_status forces(mlb_ctx *c, bool sums = false)
{
    mlb_status st = forces_pass1(c, sums);
    if (st != MLB_OK) return st;
    return sweeps(c);
}

// buffers for pass 2: u* where the last sweep left it
mlbi_buffers pass2_buffers(const mlb_ctx *c)
{
    mlbi_buffers b = c->b;
    if (c->pst_final) b.pst = c->pst_final;
    return b;
}

// the column attraction of the moments into b.attr (p.attr_r > 0)
mlb_status attraction(mlb_ctx *c)
{
    if (use_tc_attraction(c)) MLB_CUDA(c, mlbi_launch_attraction_tc(c->p, c->b, c->tc, c->stream));
    else MLB_CUDA(c, mlbi_launch_attraction(c->p, c->b, c->stream));
    return MLB_OK;
}

mlb_status forces_pass1(mlb_ctx *c, bool sums)
{
    if (c->p.local_g) {
        Timed t(c, K_MOMENTS);
        MLB_CUDA(c, mlbi_launch_moments_g(c->p, c->b, c->cur, c->stream, sums));
    } else {
        { Timed t(c, K_MOMENTS); MLB_CUDA(c, mlbi_launch_moments(c->p, c->b, c->cur, c->stream, sums)); }
        { Timed t(c, K_GFIELD); MLB_CUDA(c, mlbi_launch_gfield(c->p, c->b, c->stream)); }
    }
    if (c->p.attr_r) {
        Timed t(c, K_ATTRACTION);
        const mlb_status st = attraction(c);
        if (st != MLB_OK) return st;
    }
    if (c->surr && c->surr_active) {
        // the network's F^hc into attr; every surr_every steps the exact pass 1
        // runs instead and the network is checked against it
        { Timed t(c, K_SURROGATE); MLB_CUDA(c, mlbi_net_force_from_moments(c->surr, c->b.mom, c->b.attr, c->stream)); }
        if (c->step % c->surr_every != 0) {
            mlbi_params q = c->p;
            q.hc_from_attr = 1;
            Timed t(c, K_PASS1);
            MLB_CUDA(c, mlbi_launch_pass1(q, c->b, c->stream));
            return MLB_OK;
        }
        { Timed t(c, K_PASS1); MLB_CUDA(c, mlbi_launch_pass1(c->p, c->b, c->stream)); }
        double sums[2] = {0.0, 0.0};
        MLB_CUDA(c, mlbi_force_error((long long)c->p.S * c->p.N, c->b.attr, c->b.frest, c->surr_sums, c->stream));
        MLB_CUDA(c, cudaMemcpyAsync(sums, c->surr_sums, sizeof sums, cudaMemcpyDeviceToHost, c->stream));
        MLB_CUDA(c, cudaStreamSynchronize(c->stream));
        if (mlbi_net_timed_out(c->surr)) return fail(c, MLB_ETIMEOUT, "the surrogate's tensor-core kernel gave up a wait");
        c->surr_err = sums[1] > 0.0 ? std::sqrt(sums[0] / sums[1]) : (sums[0] > 0.0 ? 1.0 : 0.0);
        ++c->surr_rechecks;
        if (!(c->surr_err <= c->surr_bound)) {
            c->surr_active = false;
            ++c->surr_rejections;
            ++c->version;
        }
        return MLB_OK;
    }
    { Timed t(c, K_PASS1); MLB_CUDA(c, mlbi_launch_pass1(c->p, c->b, c->stream)); }
    return MLB_OK;
}

// pass 2 and the collision as two launches (else one fused launch)
bool split_collide(const mlb_ctx *c)
{
    return (c->desc.flags & MLB_SPLIT_COLLIDE) || !mlbi_pass2_collide_supported(c->p) || c->tuned_split == 1;
}

// pass 2, collision and streaming of one step (after forces())
mlb_status advance(mlb_ctx *c)
{
    const mlbi_buffers b = pass2_buffers(c);
    if (split_collide(c)) {
        { Timed t(c, K_PASS2); MLB_CUDA(c, mlbi_launch_pass2(c->p, b, nullptr, c->stream)); }
        { Timed t(c, K_COLLIDE); MLB_CUDA(c, mlbi_launch_collide(c->p, b, c->cur, c->stream)); }
    } else {
        Timed t(c, K_PASS2_COLLIDE);
        MLB_CUDA(c, mlbi_launch_pass2_collide(c->p, b, c->cur, c->stream));
    }
    return MLB_OK;
}

}  // namespace

extern "C" {

const char *mlb_status_string(mlb_status s)
{
    switch (s) {
    case MLB_OK: return "ok";
    case MLB_EINVAL: return "invalid argument";
    case MLB_ENOMEM: return "out of device memory";
    case MLB_ECUDA: return "CUDA error";
    case MLB_ENUMERIC: return "numeric fault";
    case MLB_ETIMEOUT: return "device wait timed out";
    case MLB_ESTATE: return "context not usable";
    }
    return "unknown status";
}

mlb_status mlb_velocity_set(int32_t *cv, double *w)
{
    static const int C[MLBI_Q][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                                      {0, 0, 1},  {0, 0, -1}, {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                                      {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                      {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    for (int i = 0; i < MLBI_Q; ++i) {
        if (cv)
            for (int k = 0; k < 3; ++k) cv[3 * i + k] = C[i][k];
        if (w) w[i] = i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
    return MLB_OK;
}

mlb_status mlb_create(const mlb_lattice_desc *d, mlb_ctx **out)
{
    if (!d || !out) return MLB_EINVAL;
    *out = nullptr;
    mlb_ctx *c = new (std::nothrow) mlb_ctx();
    if (!c) return MLB_ENOMEM;
    c->desc = *d;
    if (c->desc.kappa == 0.0) c->desc.kappa = 0.5;
    auto bad = [&](const char *msg) {
        c->err = msg;
        *out = c;          // the caller can read the message, then destroy
        return MLB_EINVAL;
    };
    if (d->nx < 1 || d->ny < 1 || d->nz < 1) return bad("extents must be >= 1");
    if (d->nspecies < 1 || d->nspecies > MLB_MAX_SPECIES) return bad("nspecies must be 1..4");
    if (d->wall_axis < -1 || d->wall_axis > 2) return bad("wall_axis must be -1, 0, 1 or 2");
    if (!(d->tau > 0.5) || !std::isfinite(d->tau)) return bad("tau must be finite and > 1/2");
    if (!(std::fabs(d->kT - kCs2) < 1e-12)) return bad("kT must be 1/3 (D3Q19 lattice units)");
    if (!(c->desc.kappa >= 0.0) || !std::isfinite(c->desc.kappa)) return bad("kappa must be >= 0");
    if (d->flags & ~(MLB_DRAG_ONLY | MLB_FORCE_EXPLICIT | MLB_SPLIT_COLLIDE | MLB_MEANFIELD_BF16 |
                     MLB_MEANFIELD_BF16_1PASS))
        return bad("unknown flag bits");
    if ((d->flags & MLB_MEANFIELD_BF16_1PASS) && !(d->flags & MLB_MEANFIELD_BF16))
        return bad("MLB_MEANFIELD_BF16_1PASS needs MLB_MEANFIELD_BF16");
    if (d->wall_axis >= 0) {
        if (d->wall_u_lo[d->wall_axis] != 0.0 || d->wall_u_hi[d->wall_axis] != 0.0)
            return bad("wall velocities must be tangential to the wall");
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(d->wall_u_lo[k]) || !std::isfinite(d->wall_u_hi[k]) ||
                std::fabs(d->wall_u_lo[k]) >= 0.5 || std::fabs(d->wall_u_hi[k]) >= 0.5)
                return bad("wall velocities must be finite and below 0.5");
    }
    if ((bool)d->dev_alloc != (bool)d->dev_free) return bad("dev_alloc and dev_free must be given together");
    const long long N = (long long)d->nx * d->ny * d->nz;
    // site indices are 32-bit on the device (the largest lattice that fits in
    // memory is well below this)
    if (N >= (1ll << 31)) return bad("lattice too large: nx * ny * nz must be below 2^31");
    if (d->nz > 65535 || d->ny > 65535 * 4) return bad("ny must be <= 262140 and nz <= 65535");
    if ((long long)d->nx * d->ny >= (1ll << 30)) return bad("nx * ny must be below 2^30");
    const int S = d->nspecies;

    mlbi_params &p = c->p;
    p.nx = d->nx; p.ny = d->ny; p.nz = d->nz; p.S = S; p.N = N;
    p.wall_axis = d->wall_axis;
    p.drag_only = (d->flags & MLB_DRAG_ONLY) ? 1 : 0;
    p.semi_implicit = (d->flags & MLB_FORCE_EXPLICIT) ? 0 : 1;
    p.omega = (float)(1.0 / d->tau);
    p.src_scale = p.semi_implicit ? (float)(1.0 - 0.5 / d->tau) : 1.0f;
    for (int k = 0; k < 3; ++k) {
        p.wall_lo[k] = (float)d->wall_u_lo[k];
        p.wall_hi[k] = (float)d->wall_u_hi[k];
    }

    if (d->stream) {
        c->stream = (cudaStream_t)d->stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            c->err = std::string("cudaStreamCreate: ") + cudaGetErrorString(e);
            *out = c;
            return MLB_ECUDA;
        }
        c->own_stream = true;
    }

    // one slab for every buffer
    const int npairs = S * (S + 1) / 2;
    size_t sz_f = align256(sizeof(float) * (size_t)S * MLBI_Q * N);
    size_t sz_v4 = align256(sizeof(float4) * (size_t)S * N);
    size_t sz_dg = align256(sizeof(float) * (size_t)npairs * N);
    size_t sz_tab = align256(sizeof(mlbi_entry) * 2 * kTableCap);
    size_t sz_stage = align256(sizeof(double) * (size_t)S * 4 * N);
    size_t sz_part = align256(sizeof(double) * MLBI_RED_BLOCKS * (S + 3));
    size_t sz_sums = align256(sizeof(double) * (S + 3));
    size_t sz_flags = 256;
    c->slab_bytes = 2 * sz_f + 6 * sz_v4 + sz_dg + sz_tab + sz_stage + sz_part + sz_sums + sz_flags;
    if (d->dev_alloc) {
        c->slab = d->dev_alloc(c->slab_bytes, d->alloc_user);
        if (!c->slab) {
            c->err = "dev_alloc returned NULL";
            *out = c;
            return MLB_ENOMEM;
        }
    } else {
        cudaError_t e = cudaMalloc(&c->slab, c->slab_bytes);
        if (e != cudaSuccess) {
            c->slab = nullptr;
            c->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
            *out = c;
            return MLB_ENOMEM;
        }
    }
    char *q = (char *)c->slab;
    c->b.f[0] = (float *)q; q += sz_f;
    c->b.f[1] = (float *)q; q += sz_f;
    c->b.mom = (float4 *)q; q += sz_v4;
    c->b.frest = (float4 *)q; q += sz_v4;
    c->b.pst = (float4 *)q; q += sz_v4;
    c->b.acc = (float4 *)q; q += sz_v4;
    c->b.attr = (float4 *)q; q += sz_v4;
    c->b.fext = (float4 *)q; q += sz_v4;
    c->b.dg = (float *)q; q += sz_dg;
    c->b.table = (const mlbi_entry *)q; q += sz_tab;
    c->b.stage = (double *)q; q += sz_stage;
    c->b.partial = (double *)q; q += sz_part;
    c->b.sums = (double *)q; q += sz_sums;
    c->b.flags = (unsigned int *)q;
    c->b.first_bad = (unsigned long long *)(q + 64);      // in the flags block (256 bytes)
    c->b.maps = &c->maps;
    encode_maps(c);
    cudaError_t e = cudaMemsetAsync(c->b.flags, 0, sizeof(unsigned int), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->b.fext, 0, sz_v4, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        c->err = std::string("initial memset: ") + cudaGetErrorString(e);
        c->failed = true;
        *out = c;
        return MLB_ECUDA;
    }
    c->nref.assign(S, 0.0);
    *out = c;
    return MLB_OK;
}

mlb_status mlb_set_species(mlb_ctx *c, const double *sigma, const double *mass)
{
    MLB_GUARD(c);
    if (!sigma || !mass) return fail(c, MLB_EINVAL, "sigma and mass are required");
    const int S = c->desc.nspecies;
    for (int a = 0; a < S; ++a) {
        if (!std::isfinite(sigma[a]) || sigma[a] < 1.0 || sigma[a] > 64.0)
            return fail(c, MLB_EINVAL, "sigma[%d] = %g must lie in [1, 64] lattice units", a, sigma[a]);
        if (mass[a] != 1.0) return fail(c, MLB_EINVAL, "mass[%d] = %g: every mass must be 1", a, mass[a]);
    }
    std::vector<double> old_s = c->sigma, old_m = c->mass;
    c->sigma.assign(sigma, sigma + S);
    c->mass.assign(mass, mass + S);
    if (c->eps.empty()) {
        c->eps.assign(S * S, 0.0);
        c->lambda_c.assign(S * S, 1.0);
    }
    mlb_status st = rebuild(c);
    if (st != MLB_OK) {
        c->sigma = old_s;
        c->mass = old_m;
        return st;
    }
    c->species_set = true;
    return MLB_OK;
}

mlb_status mlb_set_interactions(mlb_ctx *c, const double *eps, const double *lambda_c)
{
    MLB_GUARD(c);
    if (!c->species_set) return fail(c, MLB_ESTATE, "call mlb_set_species first");
    const int S = c->desc.nspecies;
    std::vector<double> e(S * S, 0.0), l(S * S, 1.0);
    if (eps) {
        if (!lambda_c) return fail(c, MLB_EINVAL, "lambda_c is required with eps");
        for (int a = 0; a < S; ++a)
            for (int b = 0; b < S; ++b) {
                const double x = eps[a * S + b], y = lambda_c[a * S + b];
                if (!std::isfinite(x) || x < 0.0 || x != eps[b * S + a])
                    return fail(c, MLB_EINVAL, "eps must be finite, >= 0 and symmetric (entry %d,%d)", a, b);
                if (!std::isfinite(y) || y < 1.0 || y > 16.0 || y != lambda_c[b * S + a])
                    return fail(c, MLB_EINVAL, "lambda_c must be symmetric and in [1, 16] (entry %d,%d)", a, b);
                e[a * S + b] = x;
                l[a * S + b] = y;
            }
    }
    std::vector<double> oe = c->eps, ol = c->lambda_c;
    c->eps = e;
    c->lambda_c = l;
    mlb_status st = rebuild(c);
    if (st != MLB_OK) {
        c->eps = oe;
        c->lambda_c = ol;
        rebuild(c);
    }
    return st;
}

mlb_status mlb_set_fields(mlb_ctx *c, const double *n, const double *u)
{
    MLB_GUARD(c);
    if (!c->species_set) return fail(c, MLB_ESTATE, "call mlb_set_species first");
    if (!n) return fail(c, MLB_EINVAL, "n is required");
    const int S = c->desc.nspecies;
    const long long N = c->p.N;
    // upload, then check and sum on the device; the staging buffer is scratch,
    // so a rejected field leaves the state as it was
    double *dn = c->b.stage;
    double *du = u ? c->b.stage + (size_t)S * N : nullptr;
    double v3[MLBI_MAXS];
    for (int a = 0; a < S; ++a) v3[a] = kPi / 6.0 * c->sigma[a] * c->sigma[a] * c->sigma[a];
    MLB_CUDA(c, cudaMemcpyAsync(dn, n, sizeof(double) * S * N, cudaMemcpyHostToDevice, c->stream));
    if (u) MLB_CUDA(c, cudaMemcpyAsync(du, u, sizeof(double) * S * 3 * N, cudaMemcpyHostToDevice, c->stream));
    MLB_CUDA(c, mlbi_launch_field_check(c->p, c->b, dn, du, v3, c->stream));
    double sums[MLBI_MAXS];
    unsigned long long bad[3];
    MLB_CUDA(c, cudaMemcpyAsync(sums, c->b.sums, sizeof(double) * S, cudaMemcpyDeviceToHost, c->stream));
    MLB_CUDA(c, cudaMemcpyAsync(bad, c->b.first_bad, sizeof bad, cudaMemcpyDeviceToHost, c->stream));
    MLB_CUDA(c, cudaStreamSynchronize(c->stream));
    constexpr unsigned long long kNone = ~0ull;
    if (bad[0] != kNone)
        return fail(c, MLB_EINVAL, "n[%d][%lld] = %g is not a density", (int)(bad[0] / N), (long long)(bad[0] % N),
                    n[bad[0]]);
    if (bad[1] != kNone) {
        double xi3 = 0.0;
        for (int a = 0; a < S; ++a) xi3 += v3[a] * n[a * N + (long long)bad[1]];
        return fail(c, MLB_EINVAL, "packing xi3 = %g >= 1 at site %lld", xi3, (long long)bad[1]);
    }
    if (bad[2] != kNone)
        return fail(c, MLB_EINVAL, "velocity entry %lld = %g must be finite with |u| < 1", (long long)bad[2], u[bad[2]]);
    std::vector<double> mean(S, 0.0);
    for (int a = 0; a < S; ++a) mean[a] = sums[a] / (double)N;
    std::vector<double> old = c->nref;
    for (int a = 0; a < S; ++a) c->nref[a] = (double)(float)mean[a];
    mlb_status st = rebuild(c);
    if (st != MLB_OK) {
        c->nref = old;
        return st;
    }
    MLB_CUDA(c, mlbi_launch_init(c->p, c->b, c->cur, dn, du, c->stream));
    MLB_CUDA(c, cudaStreamSynchronize(c->stream));
    c->fields_set = true;
    c->step = 0;
    return MLB_OK;
}

mlb_status mlb_set_external_force(mlb_ctx *c, const double *fext)
{
    MLB_GUARD(c);
    const int S = c->desc.nspecies;
    const long long N = c->p.N;
    if (!fext) {
        c->p.has_fext = 0;
        ++c->version;
        return MLB_OK;
    }
    for (long long k = 0; k < (long long)S * 3 * N; ++k)
        if (!std::isfinite(fext[k])) return fail(c, MLB_EINVAL, "fext entry %lld is not finite", k);
    MLB_CUDA(c, cudaMemcpyAsync(c->b.stage, fext, sizeof(double) * S * 3 * N, cudaMemcpyHostToDevice, c->stream));
    MLB_CUDA(c, mlbi_launch_import_fext(c->p, c->b, c->b.stage, c->stream));
    MLB_CUDA(c, cudaStreamSynchronize(c->stream));
    c->p.has_fext = 1;
    ++c->version;
    return MLB_OK;
}

mlb_status mlb_set_predictor_sweeps(mlb_ctx *c, int32_t sweeps)
{
    MLB_GUARD(c);
    if (sweeps < 1 || sweeps > 8) return fail(c, MLB_EINVAL, "predictor sweeps must be 1..8");
    if (!c->p.semi_implicit && sweeps != 1)
        return fail(c, MLB_EINVAL, "predictor sweeps need the semi-implicit forcing (MLB_FORCE_EXPLICIT is set)");
    if (sweeps > 1 && !c->pst2) {
        const size_t bytes = sizeof(float4) * (size_t)c->p.S * c->p.N;
        void *ptr = nullptr;
        if (c->desc.dev_alloc) {
            ptr = c->desc.dev_alloc(bytes, c->desc.alloc_user);
        } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
            ptr = nullptr;
        }
        if (!ptr) return fail(c, MLB_ENOMEM, "could not allocate the second predictor buffer (%zu bytes)", bytes);
        c->pst2 = (float4 *)ptr;
    }
    c->sweeps = sweeps;
    ++c->version;
    return MLB_OK;
}

mlb_status mlb_step(mlb_ctx *c, int64_t nsteps)
{
    MLB_GUARD(c);
    mlb_status st = require_ready(c);
    if (st != MLB_OK) return st;
    if (nsteps < 0) return fail(c, MLB_EINVAL, "nsteps must be >= 0");
    for (int64_t t = 0; t < nsteps; ++t) {
        st = forces(c);
        if (st != MLB_OK) return st;
        st = advance(c);
        if (st != MLB_OK) return st;
        c->cur ^= 1;
        ++c->step;
    }
    return MLB_OK;
}

mlb_status mlb_step_monitored(mlb_ctx *c, double *sums)
{
    MLB_GUARD(c);
    mlb_status st = require_ready(c);
    if (st != MLB_OK) return st;
    if (!sums) return fail(c, MLB_EINVAL, "sums is required");
    const int S = c->desc.nspecies;
    st = forces(c, true);                          // the moment pass also sums the state
    if (st != MLB_OK) return st;
    MLB_CUDA(c, cudaMemcpyAsync(sums, c->b.sums, sizeof(double) * (S + 3), cudaMemcpyDeviceToHost, c->stream));
    st = advance(c);
    if (st != MLB_OK) return st;
    c->cur ^= 1;
    ++c->step;
    return MLB_OK;
}

int32_t mlb_launches_per_step(const mlb_ctx *c)
{
    if (!c) return 0;
    return (c->p.local_g ? 1 : 2) + (split_collide(c) ? 3 : 2) + (c->p.attr_r ? 1 : 0) +
           (c->surr && c->surr_active ? 4 : 0) + (c->p.semi_implicit ? c->sweeps - 1 : 0);
}

const char *mlb_kernel_name(int32_t k)
{
    return (k >= 0 && k < K_NKINDS) ? kKernelNames[k] : "";
}

mlb_status mlb_profile_enable(mlb_ctx *c, int32_t enable)
{
    MLB_GUARD(c);
    c->profiling = enable != 0;
    return MLB_OK;
}

int32_t mlb_profile_read(mlb_ctx *c, double *ms, int64_t *launches, int32_t max_kernels)
{
    if (!c || c->failed) return -1;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return -1;
    for (size_t k = 0; k < c->ev_used; ++k) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, c->ev_pool[2 * k], c->ev_pool[2 * k + 1]) == cudaSuccess) {
            c->prof_ms[c->ev_kind[k]] += t;
            c->prof_count[c->ev_kind[k]] += 1;
        }
    }
    c->ev_used = 0;
    for (int k = 0; k < K_NKINDS && k < max_kernels; ++k) {
        if (ms) ms[k] = c->prof_ms[k];
        if (launches) launches[k] = c->prof_count[k];
        c->prof_ms[k] = 0.0;
        c->prof_count[k] = 0;
    }
    return K_NKINDS;
}

mlb_status mlb_synchronize(mlb_ctx *c)
{
    MLB_GUARD(c);
    MLB_CUDA(c, cudaStreamSynchronize(c->stream));
    return check_flags(c);
}

mlb_status mlb_get_moments(mlb_ctx *c, double *n, double *u)
{
    MLB_GUARD(c);
    mlb_status st = require_ready(c);
    if (st != MLB_OK) return st;
    const int S = c->desc.nspecies;
    const long long N = c->p.N;
    double *sn = c->b.stage, *su = c->b.stage + (size_t)S * N;
    MLB_CUDA(c, mlbi_launch_moments(c->p, c->b, c->cur, c->stream));
    MLB_CUDA(c, mlbi_launch_export_moments(c->p, c->b, sn, su, c->stream));
    if (n) MLB_CUDA(c, cudaMemcpyAsync(n, sn, sizeof(double) * S * N, cudaMemcpyDeviceToHost, c->stream));
    if (u) MLB_CUDA(c, cudaMemcpyAsync(u, su, sizeof(double) * S * 3 * N, cudaMemcpyDeviceToHost, c->stream));
    MLB_CUDA(c, cudaStreamSynchronize(c->stream));
    return check_flags(c);
}

mlb_status mlb_get_acceleration(mlb_ctx *c, double *acc)
{
    MLB_GUARD(c);
    mlb_status st = require_ready(c);
    if (st != MLB_OK) return st;
    if (!acc) return fail(c, MLB_EINVAL, "acc is required");
    const int S = c->desc.nspecies;
    const long long N = c->p.N;
    st = forces(c);
    if (st != MLB_OK) return st;
    MLB_CUDA(c, mlbi_launch_pass2(c->p, pass2_buffers(c), c->b.stage, c->stream));
    MLB_CUDA(c, cudaMemcpyAsync(acc, c->b.stage, sizeof(double) * S * 3 * N, cudaMemcpyDeviceToHost, c->stream));
    MLB_CUDA(c, cudaStreamSynchronize(c->stream));
    return check_flags(c);
}

mlb_status mlb_conservation(mlb_ctx *c, double *mass, double *mom)
{
    MLB_GUARD(c);
    mlb_status st = require_ready(c);
    if (st != MLB_OK) return st;
    const int S = c->desc.nspecies;
    double h[MLBI_MAXS + 3];
    MLB_CUDA(c, mlbi_launch_pop_sums(c->p, c->b, c->cur, c->stream));
    MLB_CUDA(c, cudaMemcpyAsync(h, c->b.sums, sizeof(double) * (S + 3), cudaMemcpyDeviceToHost, c->stream));
    MLB_CUDA(c, cudaStreamSynchronize(c->stream));
    st = check_flags(c);
    if (st != MLB_OK) return st;
    for (int k = 0; k < S + 3; ++k)
        if (!std::isfinite(h[k])) return fail(c, MLB_ENUMERIC, "non-finite populations met (the state diverged)");
    if (mass)
        for (int a = 0; a < S; ++a) mass[a] = h[a];
    if (mom)
        for (int k = 0; k < 3; ++k) mom[k] = h[S + k];
    return MLB_OK;
}

mlb_status mlb_get_populations(mlb_ctx *c, float *f_host, double *nref, int64_t *step)
{
    MLB_GUARD(c);
    mlb_status st = require_ready(c);
    if (st != MLB_OK) return st;
    const int S = c->desc.nspecies;
    const long long N = c->p.N;
    if (f_host)
        MLB_CUDA(c, cudaMemcpyAsync(f_host, c->b.f[c->cur], sizeof(float) * S * MLBI_Q * N, cudaMemcpyDeviceToHost,
                                    c->stream));
    MLB_CUDA(c, cudaStreamSynchronize(c->stream));
    if (nref)
        for (int a = 0; a < S; ++a) nref[a] = c->nref[a];
    if (step) *step = c->step;
    return MLB_OK;
}

mlb_status mlb_set_populations(mlb_ctx *c, const float *f_host, const double *nref, int64_t step)
{
    MLB_GUARD(c);
    if (!c->species_set) return fail(c, MLB_ESTATE, "call mlb_set_species first");
    if (!f_host || !nref) return fail(c, MLB_EINVAL, "f_host and nref are required");
    const int S = c->desc.nspecies;
    const long long N = c->p.N;
    for (int a = 0; a < S; ++a)
        if (!std::isfinite(nref[a]) || nref[a] < 0.0 || (double)(float)nref[a] != nref[a])
            return fail(c, MLB_EINVAL, "nref[%d] must be a non-negative FP32-representable value", a);
    for (long long k = 0; k < (long long)S * MLBI_Q * N; ++k)
        if (!std::isfinite(f_host[k])) return fail(c, MLB_EINVAL, "population %lld is not finite", k);
    std::vector<double> old = c->nref;
    c->nref.assign(nref, nref + S);
    mlb_status st = rebuild(c);
    if (st != MLB_OK) {
        c->nref = old;
        return st;
    }
    MLB_CUDA(c, cudaMemcpyAsync(c->b.f[c->cur], f_host, sizeof(float) * S * MLBI_Q * N, cudaMemcpyHostToDevice,
                                c->stream));
    MLB_CUDA(c, cudaStreamSynchronize(c->stream));
    c->fields_set = true;
    c->step = step;
    return MLB_OK;
}

const char *mlb_last_error(const mlb_ctx *c)
{
    if (!c) return "null context";
    return c->err.c_str();
}

mlb_status mlb_autotune(mlb_ctx *c, int32_t trials, int32_t *zchunk_out, int32_t *fused_out)
{
    MLB_GUARD(c);
    mlb_status st = require_ready(c);
    if (st != MLB_OK) return st;
    if (trials < 1) return fail(c, MLB_EINVAL, "trials must be >= 1");
    const bool prof = c->profiling;
    c->profiling = false;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MLB_CUDA(c, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(c, MLB_ECUDA, "cudaEventCreate failed");
    }
    std::vector<int> zs;
    for (int z : {4, 8, 12, 16, 32})
        if (z <= c->desc.nz) zs.push_back(z);
    if (zs.empty()) zs.push_back(c->desc.nz);
    const bool can_fuse = !(c->desc.flags & MLB_SPLIT_COLLIDE) && mlbi_pass2_collide_supported(c->p);
    float best = -1.f;
    int best_z = c->p.zchunk, best_split = c->tuned_split;
    for (int split = can_fuse ? 0 : 1; split <= 1 && st == MLB_OK; ++split) {
        c->tuned_split = can_fuse ? split : -1;
        for (int z : zs) {
            c->p.zchunk = z;
            // one untimed pass, then `trials` timed ones; cur is not advanced,
            // so every pass reads the same f[cur] and the state is untouched
            for (int t = 0; t <= trials && st == MLB_OK; ++t) {
                if (t == 1) cudaEventRecord(e0, c->stream);
                st = forces(c);
                if (st == MLB_OK) st = advance(c);
            }
            if (st != MLB_OK) break;
            cudaEventRecord(e1, c->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                st = fail(c, MLB_ECUDA, "autotune: %s", cudaGetErrorString(cudaGetLastError()));
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (best < 0.f || ms < best) {
                best = ms;
                best_z = z;
                best_split = c->tuned_split;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->profiling = prof;
    c->tuned_zchunk = best_z;
    c->p.zchunk = best_z;
    c->tuned_split = best_split;
    ++c->version;
    if (st != MLB_OK) return st;
    if (zchunk_out) *zchunk_out = best_z;
    if (fused_out) *fused_out = split_collide(c) ? 0 : 1;
    return check_flags(c);
}

void mlb_destroy(mlb_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->slab) {
        if (c->desc.dev_free) c->desc.dev_free(c->slab, c->desc.alloc_user);
        else cudaFree(c->slab);
    }
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    if (c->surr_sums) cudaFree(c->surr_sums);
    ctx_free(c, c->pst2);
    ctx_free(c, c->tc_mem);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

mlb_status mlb_get_rest_force(mlb_ctx *c, double *force)
{
    MLB_GUARD(c);
    mlb_status st = require_ready(c);
    if (st != MLB_OK) return st;
    if (!force) return fail(c, MLB_EINVAL, "force is required");
    const bool active = c->surr_active, prof = c->profiling;
    c->surr_active = false;                      // the exact force
    c->profiling = false;
    st = forces(c);
    c->surr_active = active;
    c->profiling = prof;
    if (st != MLB_OK) return st;
    const size_t bytes = sizeof(double) * 3 * c->p.S * c->p.N;
    MLB_CUDA(c, mlbi_launch_export_vec(c->p, c->b.frest, c->b.stage, c->stream));
    MLB_CUDA(c, cudaMemcpyAsync(force, c->b.stage, bytes, cudaMemcpyDeviceToHost, c->stream));
    MLB_CUDA(c, cudaStreamSynchronize(c->stream));
    return check_flags(c);
}

mlb_status mlb_attach_surrogate(mlb_ctx *c, mlb_net *net, int32_t recheck_every, double bound)
{
    MLB_GUARD(c);
    if (!net) {
        c->surr = nullptr;
        c->surr_active = false;
        ++c->version;
        return MLB_OK;
    }
    if (!c->species_set) return fail(c, MLB_ESTATE, "call mlb_set_species first");
    if (c->p.S != 2) return fail(c, MLB_EINVAL, "the surrogate serves binary mixtures");
    if (c->desc.wall_axis != -1) return fail(c, MLB_EINVAL, "the surrogate serves periodic lattices");
    if (c->p.has_attraction) return fail(c, MLB_EINVAL, "the surrogate replaces the hard core only: no tails");
    if (c->p.drag_only) return fail(c, MLB_EINVAL, "the surrogate needs the default velocity exchange");
    if (c->p.tile_r != 1 && c->p.tile_r != 2)
        return fail(c, MLB_EINVAL, "contact shells of reach %d exceed the network's 5^3 field", c->p.tile_r);
    if (!mlbi_net_matches(net, c->desc.nx, c->desc.ny, c->desc.nz))
        return fail(c, MLB_EINVAL, "the network was created for another lattice size");
    if (recheck_every < 1 || !(bound > 0.0) || !std::isfinite(bound))
        return fail(c, MLB_EINVAL, "recheck_every must be >= 1 and bound > 0");
    if (!c->surr_sums) MLB_CUDA(c, cudaMalloc(&c->surr_sums, 2 * sizeof(double)));
    c->surr = net;
    c->surr_every = recheck_every;
    c->surr_bound = bound;
    c->surr_active = true;
    c->surr_err = -1.0;
    c->surr_rechecks = c->surr_rejections = 0;
    ++c->version;
    return MLB_OK;
}

mlb_status mlb_surrogate_status(mlb_ctx *c, int32_t *active, double *last_error, int64_t *rechecks,
                                int64_t *rejections)
{
    if (!c) return MLB_EINVAL;
    if (active) *active = (c->surr && c->surr_active) ? 1 : 0;
    if (last_error) *last_error = c->surr_err;
    if (rechecks) *rechecks = c->surr_rechecks;
    if (rejections) *rejections = c->surr_rejections;
    return MLB_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batched ensemble
struct mlb_batch {
    std::vector<mlb_ctx *> m;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaGraphExec_t exec = nullptr;
    std::vector<uint64_t> version;            // members' settings at the capture
    std::vector<int> cur;                     // members' buffer parity at the capture
    cudaEvent_t cap_fork = nullptr, join = nullptr;
    std::vector<cudaEvent_t> cap_done, pre;   // per member: capture join, order before a launch
    // grouped launches: members that take the same grouped kernels step by one
    // launch per stage (mlbi_group); the others by their own launches
    int lanes = 1;                            // 0: no grouping; else lanes per group
    long long group_max_sites = 1ll << 17;    // larger members step by their own launches
    std::vector<mlbi_group> groups;           // one per lane
    std::vector<std::vector<int>> group_members;
    void *gmem = nullptr;                     // device: member tables and block tables of every lane
    std::vector<cudaEvent_t> lane_ev;         // per lane: lane done
    cudaEvent_t attr_fork = nullptr;
    // mlb_batch_synchronize: every member's flag word gathered by one kernel
    const unsigned int **flag_ptrs = nullptr;  // device [n]
    unsigned int *flag_words = nullptr;         // device [n]
    unsigned int *flag_host = nullptr;          // pinned host [n]
    bool failed = false;
    std::string err;
};

namespace {

mlb_status batch_fail(mlb_batch *b, mlb_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    b->err = buf;
    if (s == MLB_ECUDA) b->failed = true;
    return s;
}

// whether a member can step inside a grouped launch (the fused pass 2 +
// collision is bitwise the split pair, so a tuned split does not exclude it)
bool groupable(const mlb_batch *b, const mlb_ctx *c)
{
    return c->p.N <= b->group_max_sites && c->sweeps == 1 && !(c->surr && c->surr_active) &&
           !(c->desc.flags & MLB_SPLIT_COLLIDE) && mlbi_group_supported(c->p, c->b);
}

void free_groups(mlb_batch *b)
{
    if (b->gmem) {
        cudaStreamSynchronize(b->stream);     // a graph still in flight may read the tables
        cudaFree(b->gmem);
        b->gmem = nullptr;
    }
    b->groups.clear();
    b->group_members.clear();
}

// Partition the members by (species, shell reach, drag mode) among those that
// can be grouped, and each such group into `lanes` lanes (members dealt in
// order of size, so the lanes carry similar work); write each lane's member
// table and per-stage block tables (larger members first) to one device
// allocation.
mlb_status build_groups(mlb_batch *b)
{
    free_groups(b);
    if (b->lanes < 1) return MLB_OK;
    std::vector<std::vector<int>> sets;
    for (size_t i = 0; i < b->m.size(); ++i) {
        const mlb_ctx *c = b->m[i];
        if (!groupable(b, c)) continue;
        bool placed = false;
        for (auto &g : sets) {
            const mlbi_params &q = b->m[g[0]]->p;
            if (q.S == c->p.S && q.tile_r == c->p.tile_r && q.drag_only == c->p.drag_only) {
                g.push_back((int)i);
                placed = true;
                break;
            }
        }
        if (!placed) sets.push_back({(int)i});
    }
    for (auto &g : sets) {
        if (g.size() < 2) continue;           // one member steps as fast by its own launches
        std::stable_sort(g.begin(), g.end(), [&](int x, int y) { return b->m[x]->p.N > b->m[y]->p.N; });
        const size_t nl = std::min(g.size(), (size_t)b->lanes);
        std::vector<std::vector<int>> lanes(nl);
        for (size_t k = 0; k < g.size(); ++k) lanes[k % nl].push_back(g[k]);
        for (auto &l : lanes) b->group_members.push_back(l);
    }
    while (b->lane_ev.size() < b->group_members.size()) {
        cudaEvent_t ev = nullptr;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
            return batch_fail(b, MLB_ECUDA, "cudaEventCreate failed");
        b->lane_ev.push_back(ev);
    }
    if (b->group_members.empty()) return MLB_OK;
    // layout: per group the members, then the three block tables
    std::vector<size_t> off_mem, off_blk[3];
    std::vector<std::vector<int4>> tables[3];
    size_t bytes = 0;
    auto take = [&](size_t n) { bytes = (bytes + 255) & ~size_t(255); const size_t o = bytes; bytes += n; return o; };
    for (const auto &g : b->group_members) {
        off_mem.push_back(take(g.size() * sizeof(mlbi_member)));
        for (int k = 0; k < 3; ++k) {
            std::vector<int4> t;
            for (size_t j = 0; j < g.size(); ++j) {
                int grid[3];
                mlbi_group_grid(b->m[g[j]]->p, k, grid);
                const long long nb = (long long)grid[0] * grid[1] * grid[2];
                if (nb + (long long)t.size() > (1ll << 30)) return batch_fail(b, MLB_EINVAL, "group too large");
                for (long long q = 0; q < nb; ++q) {
                    if (k == MLBI_GROUP_MOMENTS)
                        t.push_back(make_int4((int)j, (int)q, (int)nb, 0));
                    else
                        t.push_back(make_int4((int)j, (int)(q % grid[0]), (int)(q / grid[0] % grid[1]),
                                              (int)(q / ((long long)grid[0] * grid[1]))));
                }
            }
            off_blk[k].push_back(take(t.size() * sizeof(int4)));
            tables[k].push_back(std::move(t));
        }
    }
    cudaError_t e = cudaMalloc(&b->gmem, bytes);
    if (e != cudaSuccess) {
        b->gmem = nullptr;
        return batch_fail(b, MLB_ENOMEM, "group tables: %s", cudaGetErrorString(e));
    }
    char *base = static_cast<char *>(b->gmem);
    for (size_t gi = 0; gi < b->group_members.size() && e == cudaSuccess; ++gi) {
        const auto &g = b->group_members[gi];
        std::vector<mlbi_member> mem(g.size());
        for (size_t j = 0; j < g.size(); ++j) {
            const mlb_ctx *c = b->m[g[j]];
            std::memset(static_cast<void *>(&mem[j]), 0, sizeof(mlbi_member));
            mem[j].map_f[0] = c->maps.f[0];
            mem[j].map_f[1] = c->maps.f[1];
            mem[j].map_mom = c->maps.mom;
            mem[j].map_frest = c->maps.frest;
            mem[j].p = c->p;
            mem[j].b = c->b;
            mem[j].b.maps = nullptr;
            mem[j].cur = c->cur;
        }
        e = cudaMemcpy(base + off_mem[gi], mem.data(), mem.size() * sizeof(mlbi_member), cudaMemcpyHostToDevice);
        mlbi_group grp{};
        grp.mem = reinterpret_cast<const mlbi_member *>(base + off_mem[gi]);
        for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
            e = cudaMemcpy(base + off_blk[k][gi], tables[k][gi].data(), tables[k][gi].size() * sizeof(int4),
                           cudaMemcpyHostToDevice);
            grp.blk[k] = reinterpret_cast<const int4 *>(base + off_blk[k][gi]);
            grp.nblk[k] = (int)tables[k][gi].size();
        }
        const mlbi_params &q = b->m[g[0]]->p;
        grp.S = q.S;
        grp.R = q.tile_r;
        grp.drag = q.drag_only;
        b->groups.push_back(grp);
    }
    if (e != cudaSuccess) return batch_fail(b, MLB_ECUDA, "group tables: %s", cudaGetErrorString(e));
    return MLB_OK;
}

// Capture two steps of every member into a graph.  Grouped members: per step
// one launch per stage for each lane on the lane's stream (forked from the
// batch stream), the column attractions of members that have one forked onto
// their own streams between the moments and pass 1.  The other members: fork
// from the batch stream onto each member's stream, two (forces, advance)
// pairs per member, join back.
mlb_status batch_capture(mlb_batch *b)
{
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    for (size_t i = 0; i < b->m.size(); ++i)
        if (b->m[i]->surr && b->m[i]->surr_active)
            return batch_fail(b, MLB_EINVAL, "member %zu uses a surrogate (its rechecks read back to the host)", i);
    mlb_status st = build_groups(b);
    if (st != MLB_OK) return st;
    std::vector<char> in_group(b->m.size(), 0);
    for (const auto &g : b->group_members)
        for (int i : g) in_group[i] = 1;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return batch_fail(b, MLB_ECUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
    e = cudaEventRecord(b->cap_fork, b->stream);
    // each lane on the stream of its first member
    for (size_t l = 0; l < b->groups.size() && e == cudaSuccess && st == MLB_OK; ++l) {
        const mlbi_group &g = b->groups[l];
        cudaStream_t ls = b->m[b->group_members[l][0]]->stream;
        e = cudaStreamWaitEvent(ls, b->cap_fork, 0);
        for (int odd = 0; odd < 2 && e == cudaSuccess && st == MLB_OK; ++odd) {
            e = mlbi_launch_group_moments(g, odd, ls);
            bool forked = false;
            for (int i : b->group_members[l]) {
                mlb_ctx *c = b->m[i];
                if (!c->p.attr_r || e != cudaSuccess || st != MLB_OK) continue;
                if (c->stream == ls) {
                    st = attraction(c);
                    continue;
                }
                if (!forked) e = cudaEventRecord(b->attr_fork, ls);
                forked = true;
                if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, b->attr_fork, 0);
                if (e == cudaSuccess) st = attraction(c);
                if (e == cudaSuccess && st == MLB_OK) e = cudaEventRecord(b->cap_done[i], c->stream);
                if (e == cudaSuccess && st == MLB_OK) e = cudaStreamWaitEvent(ls, b->cap_done[i], 0);
            }
            if (e == cudaSuccess && st == MLB_OK) e = mlbi_launch_group_pass1(g, ls);
            if (e == cudaSuccess && st == MLB_OK) e = mlbi_launch_group_pass2_collide(g, odd, ls);
        }
        if (e == cudaSuccess) e = cudaEventRecord(b->lane_ev[l], ls);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->lane_ev[l], 0);
    }
    for (size_t i = 0; i < b->m.size() && e == cudaSuccess && st == MLB_OK; ++i) {
        if (in_group[i]) continue;
        mlb_ctx *c = b->m[i];
        const bool prof = c->profiling;
        c->profiling = false;
        e = cudaStreamWaitEvent(c->stream, b->cap_fork, 0);
        for (int k = 0; k < 2 && e == cudaSuccess && st == MLB_OK; ++k) {
            st = forces(c);
            if (st == MLB_OK) st = advance(c);
            c->cur ^= 1;                      // two flips: back to the captured parity
        }
        c->profiling = prof;
        if (e == cudaSuccess) e = cudaEventRecord(b->cap_done[i], c->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->cap_done[i], 0);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b->stream, &g);
    if (e == cudaSuccess) e = ee;
    if (st != MLB_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        free_groups(b);
        if (st != MLB_OK) return batch_fail(b, MLB_ECUDA, "capture: member launch failed");
        return batch_fail(b, MLB_ECUDA, "capture: %s", cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->exec = nullptr;
        return batch_fail(b, MLB_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    }
    for (size_t i = 0; i < b->m.size(); ++i) {
        b->version[i] = b->m[i]->version;
        b->cur[i] = b->m[i]->cur;
    }
    return MLB_OK;
}

}  // namespace

extern "C" {

mlb_status mlb_batch_create(mlb_ctx *const *members, int32_t n, void *stream, mlb_batch **out)
{
    if (!out) return MLB_EINVAL;
    *out = nullptr;
    if (!members || n < 1) return MLB_EINVAL;
    for (int32_t i = 0; i < n; ++i) {
        if (!members[i] || members[i]->failed || !members[i]->stream) return MLB_EINVAL;
        for (int32_t j = 0; j < i; ++j)
            if (members[j] == members[i]) return MLB_EINVAL;
    }
    mlb_batch *b = new (std::nothrow) mlb_batch();
    if (!b) return MLB_ENOMEM;
    b->m.assign(members, members + n);
    b->version.assign(n, 0);
    b->cur.assign(n, -1);
    b->cap_done.assign(n, nullptr);
    b->pre.assign(n, nullptr);
    cudaError_t e = cudaSuccess;
    if (stream) {
        b->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        b->own_stream = e == cudaSuccess;
    }
    const unsigned fl = cudaEventDisableTiming;
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->cap_fork, fl);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join, fl);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->attr_fork, fl);
    for (int32_t i = 0; i < n && e == cudaSuccess; ++i) {
        e = cudaEventCreateWithFlags(&b->cap_done[i], fl);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->pre[i], fl);
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->flag_ptrs, sizeof(unsigned int *) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->flag_words, sizeof(unsigned int) * n);
    if (e == cudaSuccess) e = cudaMallocHost(&b->flag_host, sizeof(unsigned int) * n);
    if (e == cudaSuccess) {
        std::vector<const unsigned int *> ptrs(n);
        for (int32_t i = 0; i < n; ++i) ptrs[i] = members[i]->b.flags;
        e = cudaMemcpy(b->flag_ptrs, ptrs.data(), sizeof(unsigned int *) * n, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        mlb_batch_destroy(b);
        return MLB_ECUDA;
    }
    *out = b;
    return MLB_OK;
}

mlb_status mlb_batch_step(mlb_batch *b, int64_t nsteps)
{
    if (!b) return MLB_EINVAL;
    if (b->failed) return MLB_ESTATE;
    if (nsteps < 0) return batch_fail(b, MLB_EINVAL, "nsteps must be >= 0");
    for (size_t i = 0; i < b->m.size(); ++i) {
        mlb_ctx *c = b->m[i];
        if (c->failed) return batch_fail(b, MLB_ESTATE, "member %zu is in a failed state: %s", i, c->err.c_str());
        if (require_ready(c) != MLB_OK) return batch_fail(b, MLB_ESTATE, "member %zu: %s", i, c->err.c_str());
    }
    const int64_t pairs = nsteps / 2;
    if (pairs > 0) {
        bool stale = !b->exec;
        for (size_t i = 0; i < b->m.size() && !stale; ++i)
            stale = b->version[i] != b->m[i]->version || b->cur[i] != b->m[i]->cur;
        if (stale) {
            mlb_status st = batch_capture(b);
            if (st != MLB_OK) return st;
        }
        cudaError_t e = cudaSuccess;
        for (size_t i = 0; i < b->m.size() && e == cudaSuccess; ++i) {
            e = cudaEventRecord(b->pre[i], b->m[i]->stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->pre[i], 0);
        }
        for (int64_t k = 0; k < pairs && e == cudaSuccess; ++k) e = cudaGraphLaunch(b->exec, b->stream);
        if (e == cudaSuccess) e = cudaEventRecord(b->join, b->stream);
        for (size_t i = 0; i < b->m.size() && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(b->m[i]->stream, b->join, 0);
        if (e != cudaSuccess) return batch_fail(b, MLB_ECUDA, "graph launch: %s", cudaGetErrorString(e));
        for (mlb_ctx *c : b->m) c->step += 2 * pairs;
    }
    if (nsteps % 2)
        for (size_t i = 0; i < b->m.size(); ++i) {
            const mlb_status st = mlb_step(b->m[i], 1);
            if (st != MLB_OK) return batch_fail(b, st, "member %zu: %s", i, b->m[i]->err.c_str());
        }
    return MLB_OK;
}

// Waits for every member's stream (each joined into the batch stream by an
// event), then reads all members' fault flags with one gather launch and one
// copy, and reports the first member whose flags are set.
mlb_status mlb_batch_synchronize(mlb_batch *b)
{
    if (!b) return MLB_EINVAL;
    if (b->failed) return MLB_ESTATE;
    const int n = (int)b->m.size();
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        e = cudaEventRecord(b->pre[i], b->m[i]->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->pre[i], 0);
    }
    if (e == cudaSuccess) e = mlbi_launch_gather_flags(b->flag_ptrs, n, b->flag_words, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->flag_host, b->flag_words, sizeof(unsigned int) * n, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return batch_fail(b, MLB_ECUDA, "synchronize: %s", cudaGetErrorString(e));
    for (int i = 0; i < n; ++i) {
        const mlb_status st = flags_status(b->m[i], b->flag_host[i]);
        if (st != MLB_OK) return batch_fail(b, st, "member %d: %s", i, b->m[i]->err.c_str());
    }
    return MLB_OK;
}

mlb_status mlb_batch_set_grouping(mlb_batch *b, int32_t lanes, int64_t max_sites)
{
    if (!b) return MLB_EINVAL;
    if (b->failed) return MLB_ESTATE;
    if (lanes < 0 || lanes > 64) return batch_fail(b, MLB_EINVAL, "lanes must be 0..64");
    if (max_sites < 1) return batch_fail(b, MLB_EINVAL, "max_sites must be >= 1");
    if (b->lanes != lanes || b->group_max_sites != max_sites) {
        b->lanes = lanes;
        b->group_max_sites = max_sites;
        if (b->exec) {
            cudaStreamSynchronize(b->stream);
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
    }
    return MLB_OK;
}

int32_t mlb_batch_grouped_members(const mlb_batch *b)
{
    if (!b) return 0;
    int32_t n = 0;
    for (const auto &g : b->group_members) n += (int32_t)g.size();
    return n;
}

const char *mlb_batch_last_error(const mlb_batch *b)
{
    return b ? b->err.c_str() : "null batch";
}

void mlb_batch_destroy(mlb_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    free_groups(b);
    if (b->flag_ptrs) cudaFree(b->flag_ptrs);
    if (b->flag_words) cudaFree(b->flag_words);
    if (b->flag_host) cudaFreeHost(b->flag_host);
    for (cudaEvent_t e : b->lane_ev)
        if (e) cudaEventDestroy(e);
    if (b->attr_fork) cudaEventDestroy(b->attr_fork);
    if (b->cap_fork) cudaEventDestroy(b->cap_fork);
    if (b->join) cudaEventDestroy(b->join);
    for (cudaEvent_t e : b->cap_done)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : b->pre)
        if (e) cudaEventDestroy(e);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"
