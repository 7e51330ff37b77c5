// mlb_internal.h -- definitions shared by the C-ABI runtime (mlb_api.cu) and
// the sm_103a kernel units (mlb_kernels.cu, mlb_pass1.cu, mlb_pass2.cu,
// mlb_attraction.cu).  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#define MLBI_Q 19
#define MLBI_MAXS 4
#define MLBI_MAXP 10            // unordered species pairs for MLBI_MAXS species

// One stencil entry is two float4 in the table:
//   e0 = (x, y, z, packed d): a unit vector s_d or a kernel vector, and the
//        offset d packed as three signed 10-bit fields (see mlbi_pack);
//   e1 = (linear offset of d for this lattice, mask, tile offset, dz) as
//        int bits; the mask (union shells) has bit a set when d lies in the
//        shell of the pair (a, b) of the table's neighbour species b; the
//        tile offset dx + dy (32 + 2 tile_r) addresses d inside a plane of
//        the shared-memory tile of the tiled kernels.
typedef float4 mlbi_entry;

__host__ __device__ inline int mlbi_pack(int dx, int dy, int dz)
{
    return (dx + 512) | ((dy + 512) << 10) | ((dz + 512) << 20);
}
__host__ __device__ inline void mlbi_unpack(int p, int &dx, int &dy, int &dz)
{
    dx = (p & 1023) - 512;
    dy = ((p >> 10) & 1023) - 512;
    dz = ((p >> 20) & 1023) - 512;
}

struct mlbi_pair {               // unordered pair a <= b, index a*S - a(a-1)/2 + (b - a)
    int shell_start, shell_count;    // half shell: one of each +-d (entries)
    int attr_start, attr_count;      // half attraction region (entries)
    float hc_pre;                    // kT sigma_ab^2 4 pi / |S_ab|
    float vx_pre;                    // K_ab 4 pi / |S_ab|,  K_ab = 2 sigma_ab^2 sqrt(2 mu_ab kT / pi)
    float h;                         // BMCSL h_ab = sigma_a sigma_b / (sigma_a + sigma_b)
    float g_ref;                     // BMCSL contact value at the reference densities
};

struct mlbi_params {
    int nx, ny, nz, S;
    long long N;
    int wall_axis;                   // -1 periodic
    int drag_only;
    int semi_implicit;               // 1: half-force shift, 0: forward Euler
    int has_fext;
    int has_attraction;
    int npairs;
    float omega;
    float src_scale;                 // 1 - omega/2 (semi-implicit) or 1
    float nref[MLBI_MAXS];
    float xi2_coef[MLBI_MAXS];       // (pi/6) sigma^2
    float xi3_coef[MLBI_MAXS];       // (pi/6) sigma^3
    float xi2_ref, xi3_ref;
    int ball_start[MLBI_MAXS], ball_count[MLBI_MAXS];
    float ball_inv[MLBI_MAXS];
    int ushell_start[MLBI_MAXS], ushell_count[MLBI_MAXS];   // union half shells per neighbour species
    int reach;                       // largest offset component of any stencil (>= 1)
    int local_g;                     // every smoothing ball is the single site
    int tile_r;                      // reach of the union shells if the tiled kernels serve it (1..3), else 0
    int cube_mask[MLBI_MAXP];        // tile_r == 1: bit k set when half offset k of the 3x3x3 cube is in S_ab
    int attr_r;                      // reach of the attraction if the column attraction kernel serves it (1..8), else 0
    // column form of the attraction (attr_r > 0): acol_count columns (dx, dy) of the
    // half plane, one float4 each at table[acol_start] = (dx, dy, E, 0) as int bits,
    // E the largest |dz| any pair reaches on the column; their weights are float2
    // (k, dz k) per (column, pair, dz = 0..attr_r) at ((float2 *)(table + aw_start))
    int acol_start, acol_count, aw_start;
    int zchunk;                      // planes per block of the tiled kernels
    int hc_from_attr;                // 1: pass 1 skips the hard-core sums and takes attr as F^hc (surrogate)
    int pair_index[MLBI_MAXS][MLBI_MAXS];
    mlbi_pair pair[MLBI_MAXP];
    float wall_lo[3], wall_hi[3];
};

// Shared-memory z-marching tiles of the stencil passes: a ring of 2R + 2
// planes of (32 + 2R) x (ty + 2R) sites, each site S float4 fields and
// S(S+1)/2 contact-value deviations.  Tiles serve shell reach R <= 3; reach 1
// and 2 use 32 x 4 blocks, reach 3 32 x 8 blocks where they fit, else 32 x 4.
#define MLBI_MAX_TILE_BYTES (227 * 1024)
__host__ __device__ constexpr long long mlbi_tile_bytes(int S, int R, int ty)
{
    return (long long)(2 * R + 2) * (32 + 2 * R) * (ty + 2 * R) * (S * 16 + S * (S + 1) / 2 * 4);
}
// warps per SM that tiles of block height ty leave resident (the shared-memory
// bound: 228 KB per SM, 1 KB reserved per block)
__host__ __device__ constexpr long long mlbi_tile_warps(int S, int R, int ty)
{
    return (228 * 1024) / (mlbi_tile_bytes(S, R, ty) + 1024) * ty;
}
// block height of the tile for (S, R), or 0 for the global-memory passes: a
// tile that fits and leaves at least 8 resident warps per SM (one 4-warp
// block per SM is latency-bound: measured slower than the global passes for
// three species at reach 3, while one 8-warp block per SM beats them for
// two species at reach 3)
__host__ __device__ constexpr int mlbi_tile_ty(int S, int R)
{
    return R < 1 || R > 3 ? 0
         : R < 3 ? (mlbi_tile_bytes(S, R, 4) <= MLBI_MAX_TILE_BYTES && mlbi_tile_warps(S, R, 4) >= 8 ? 4 : 0)
         : mlbi_tile_bytes(S, R, 8) <= MLBI_MAX_TILE_BYTES ? 8
         : (mlbi_tile_bytes(S, R, 4) <= MLBI_MAX_TILE_BYTES && mlbi_tile_warps(S, R, 4) >= 8 ? 4 : 0);
}

// Bulk tensor (TMA) descriptors of the buffers the fused pass-2 + collision
// kernel copies plane by plane: the populations f[c] as a 4D FP32 tensor
// (x, y, z, S*19), the moments and the rest force as 5D (4 components, x,
// y, z, S).  ok = 0 (no TMA: nx not a multiple of 4, or the encode failed)
// selects the cp.async variant.
struct mlbi_maps {
    CUtensorMap f[2];
    CUtensorMap mom;
    CUtensorMap frest;
    int ok;
};

// Tables of the tensor-core attraction (mlb_attraction_tc.cu), device memory
// owned by the context: per column (dx, dy), sorted by dy then dx, the B
// operands hi and lo; the columns and the first column of every dy row; the
// BF16 hi / lo copies of n - n_ref in the layout [y][b][z / 8][x][8 planes].
struct mlbi_tc_tables {
    void *weights;                   // [ncols][hi, lo][K / 8][N][8] BF16
    int2 *cols;                      // [ncols] (dx, dy)
    int *row_start;                  // [nrows + 1]
    void *qhi, *qlo;                 // [nyp][S][nz / 8][nxp][8] BF16 each (padded, mlbi_attraction_tc_padded)
    int ncols, nrows;
    int pass3;                       // 1: compensated hi/lo product, 0: hi only
};

// Device buffers of one context (all carved from one allocation).
struct mlbi_buffers {
    float *f[2];                     // [S][19][N] populations minus w_i n_ref
    float4 *mom;                     // [S][N]  (dn, ux, uy, uz), dn = n - n_ref
    float *dg;                       // [npairs][N]  g_ab - g_ref_ab
    float4 *frest;                   // [S][N]  pass 1 -> 2: F^hc + G + F_ext
    float4 *pst;                     // [S][N]  pass 1 -> 2: (n - n_ref, u* = u + du)
    float4 *acc;                     // [S][N]  pass 2 -> collide: acceleration
    float4 *attr;                    // [S][N]  attraction G^a (column attraction kernel -> pass 1)
    float4 *fext;                    // [S][N]  external force (if any)
    const mlbi_entry *table;         // stencil entries
    double *stage;                   // [S*4*N] FP64 staging for host transfers
    double *partial;                 // [MLBI_RED_BLOCKS][S+3] FP64 block sums
    double *sums;                    // [S+3] final sums
    unsigned int *flags;             // [1] numeric fault flags
    const mlbi_maps *maps;           // host copy of the TMA descriptors (owned by the context)
    unsigned long long *first_bad;   // [3] first invalid entry of uploaded fields (n, xi3, u)
};

#define MLBI_RED_BLOCKS 1024
#define MLBI_FLAG_XI3 1u
#define MLBI_FLAG_NAN 2u
#define MLBI_FLAG_TIMEOUT 4u            // a bounded device wait gave up


// kernel launchers (one per kernel unit); each returns cudaGetLastError()
// sums: also the FP64 conservation sums of the state into b.sums (mass[S],
// mom[3]; a grid of MLBI_RED_BLOCKS blocks and the final reduction)
cudaError_t mlbi_launch_moments(const mlbi_params &p, const mlbi_buffers &b, int cur, cudaStream_t s,
                                bool sums = false);
// FP64 sums of the populations f[cur] themselves into b.sums (mass[S], mom[3];
// mlb_popsum.cuh; b.partial holds the block partials)
cudaError_t mlbi_launch_pop_sums(const mlbi_params &p, const mlbi_buffers &b, int cur, cudaStream_t s);
cudaError_t mlbi_launch_gfield(const mlbi_params &p, const mlbi_buffers &b, cudaStream_t s);
cudaError_t mlbi_launch_pass1(const mlbi_params &p, const mlbi_buffers &b, cudaStream_t s);
// one further Jacobi sweep of the half step: prev = the previous sweep's
// (n - n_ref, u*) [S][N], next receives this sweep's (must differ from prev);
// b.mom, b.dg, b.frest as left by pass 1
cudaError_t mlbi_launch_sweep(const mlbi_params &p, const mlbi_buffers &b, const float4 *prev, float4 *next,
                              cudaStream_t s);
// tensor-core attraction: whether the lattice and species suit it (S <= 2,
// reach <= 8, no walls normal to z, nz % 8 == 0), bytes of one column's B
// operands, and the launch (prep + implicit GEMM) writing b.attr
bool mlbi_attraction_tc_supported(const mlbi_params &p);
size_t mlbi_attraction_tc_column_bytes(int S);
// padded extents of the BF16 density copies (an 8-site halo in x and y, x up to whole tiles)
void mlbi_attraction_tc_padded(const mlbi_params &p, int *nxp, int *nyp);
cudaError_t mlbi_launch_attraction_tc(const mlbi_params &p, const mlbi_buffers &b, const mlbi_tc_tables &t,
                                      cudaStream_t s);
cudaError_t mlbi_launch_attraction(const mlbi_params &p, const mlbi_buffers &b, cudaStream_t s);
cudaError_t mlbi_launch_moments_g(const mlbi_params &p, const mlbi_buffers &b, int cur, cudaStream_t s,
                                  bool sums = false);
// Uploaded fields n [S][N] and u [S][3][N] (u may be NULL), FP64 in device
// memory: the per-species sums of n into b.sums[0 .. S-1], and in
// b.first_bad the first flat index of n not finite or negative, of a site with
// xi3 = sum_a v3[a] n^a >= 1, and of u not finite or |u| >= 1 (all ones where
// none; b.first_bad is reset by the launch)
cudaError_t mlbi_launch_field_check(const mlbi_params &p, const mlbi_buffers &b, const double *n, const double *u,
                                    const double *v3, cudaStream_t s);
cudaError_t mlbi_launch_pass2(const mlbi_params &p, const mlbi_buffers &b, double *acc_out, cudaStream_t s);
cudaError_t mlbi_launch_collide(const mlbi_params &p, const mlbi_buffers &b, int cur, cudaStream_t s);
// pass 2 fused with the collision and streaming of f[cur] -> f[cur ^ 1] (no acceleration
// stored); only where mlbi_pass2_collide_supported (tiled passes whose fused tile fits
// in shared memory), else cudaErrorInvalidValue
bool mlbi_pass2_collide_supported(const mlbi_params &p);
cudaError_t mlbi_launch_pass2_collide(const mlbi_params &p, const mlbi_buffers &b, int cur, cudaStream_t s);
cudaError_t mlbi_launch_init(const mlbi_params &p, const mlbi_buffers &b, int cur, const double *n,
                             const double *u, cudaStream_t s);
cudaError_t mlbi_launch_export_moments(const mlbi_params &p, const mlbi_buffers &b, double *n_out,
                                       double *u_out, cudaStream_t s);
cudaError_t mlbi_launch_import_fext(const mlbi_params &p, const mlbi_buffers &b, const double *fext,
                                    cudaStream_t s);
// float4 [S][N] (x, y, z) -> FP64 [S][3][N]
cudaError_t mlbi_launch_export_vec(const mlbi_params &p, const float4 *src, double *dst, cudaStream_t s);

// ------------------------------------------------------------------ grouped launches
// One launch of a stage steps every member of a group of independent
// lattices (mlb_batch): the members take the same kernel instantiation (same
// S, shell reach and drag mode; site-local contact values; the fused pass 2 +
// collision on bulk tensor copies), each block reads its member and tile from
// a block table, copies the member's parameters into shared memory and runs
// the stage's per-block code unchanged, so a member's arithmetic is bitwise
// that of its own launches.  Device memory; the tensor maps are the
// members' host-encoded descriptors copied to global memory.
struct mlbi_member {
    CUtensorMap map_f[2];            // populations f[0], f[1]
    CUtensorMap map_mom, map_frest;
    mlbi_params p;
    mlbi_buffers b;                  // device pointers of the member (b.maps unused)
    int cur;                         // the buffer f[cur] the member reads at the group's even steps
};
struct mlbi_group {
    const mlbi_member *mem;          // [nmem] device
    const int4 *blk[3];              // per stage: [nblk] {member, block x, block y, block z} device
    int nblk[3];                     // (moments: {member, block, blocks of the member, 0})
    int S, R, drag;                  // the shared instantiation: species, shell reach (1, 2), drag only
};
enum { MLBI_GROUP_MOMENTS = 0, MLBI_GROUP_PASS1 = 1, MLBI_GROUP_PASS2 = 2 };
// whether a member can join a group, and its stage grids (blocks per stage)
bool mlbi_group_supported(const mlbi_params &p, const mlbi_buffers &b);
void mlbi_group_grid(const mlbi_params &p, int stage, int grid[3]);
// out[i] = *flags[i] for n contexts' fault-flag words (one launch; mlb_batch)
cudaError_t mlbi_launch_gather_flags(const unsigned int *const *flags, int n, unsigned int *out, cudaStream_t s);
// odd: the group's odd step (members read f[cur ^ 1])
cudaError_t mlbi_launch_group_moments(const mlbi_group &g, int odd, cudaStream_t s);
cudaError_t mlbi_launch_group_pass1(const mlbi_group &g, cudaStream_t s);
cudaError_t mlbi_launch_group_pass2_collide(const mlbi_group &g, int odd, cudaStream_t s);

// learned surrogate of the hard-core force (mlb_surrogate.cu)
struct mlb_net;
bool mlbi_net_matches(const mlb_net *n, int nx, int ny, int nz);
// a bounded wait in the network's tensor-core kernel gave up (synchronous read)
bool mlbi_net_timed_out(mlb_net *n);
// force[S][N] = the network's F^hc from the moments' n - n_ref
cudaError_t mlbi_net_force_from_moments(mlb_net *n, const float4 *mom, float4 *force, cudaStream_t s);
// sums[0] = sum |fs - fx|^2, sums[1] = sum |fx|^2 over n4 float4 (x, y, z)
cudaError_t mlbi_force_error(long long n4, const float4 *fs, const float4 *fx, double *sums, cudaStream_t s);
