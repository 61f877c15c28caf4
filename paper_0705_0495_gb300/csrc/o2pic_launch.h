// o2pic_launch.h -- host-side launch wrappers of the libo2pic kernels.
#pragma once
#include <cuda_runtime.h>

#include "o2pic_dev.cuh"

namespace o2 {

// Launch of a time-step kernel with programmatic stream serialization (the
// kernel itself waits for its predecessor with pdl_wait()).
#ifndef O2_PDL
#define O2_PDL 1
#endif
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                            Args &&...args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = O2_PDL;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

constexpr int MAX_PUSH_SHAPES = 8;

struct LaunchCfg {
    int push_blocks;      // persistent grid of the push
    int push_per_sm;      // its blocks per SM
    int push_max_per_sm;  // the most that fit on an SM (current shape)
    int push_shape;       // index of the push's launch shape
    int push_nshapes;     // shapes compiled for this precision
    int shape_threads[MAX_PUSH_SHAPES], shape_spt[MAX_PUSH_SHAPES], shape_max_per_sm[MAX_PUSH_SHAPES];
    size_t shape_smem[MAX_PUSH_SHAPES], shape_smem_diag[MAX_PUSH_SHAPES];
    int num_sms;
    int collide_blocks;   // grid of the collision kernel (loops over the candidates)
    size_t push_smem;     // dynamic shared memory of the push (non-diag)
    size_t push_smem_diag;
    int sort_blocks;      // sum over (d, s) of sort blocks
    size_t sort_smem;     // count kernel
    size_t scatter_smem;  // scatter kernel
    int sort_col_warps;   // warps of the column scan (sum over (d, s) of bucket groups x row segments)
    const int *sort_warp_base;  // device [D*3+1]: first column-scan warp per (d, s)
    int pair_blocks_sp[NSP];          // evaluation blocks per projectile species
    const int *pair_tab_sp[NSP];      // device [(d, tile)] tables per species
    size_t field_smem;
    int maxN;             // largest cell count over discharges
    int eedf_max, fm_max; // largest histogram sizes (shared-memory copies in the push)
};

// push + absorb + null-collision MCC + births + deposit (one time step)
cudaError_t launch_push(bool fp64, bool diag, const WsPtrs &W, const void *pools,
                        int par, const LaunchCfg &L, cudaStream_t s);
cudaError_t push_configure(bool fp64, LaunchCfg &L, int num_sms);
// births of the push appended in parent order
cudaError_t launch_collide(bool fp64, const WsPtrs &W, const void *pools, int par, int blocks, cudaStream_t st);
// salt: 0 for the append after the collisions, 1 for the one after the
// sequential gas scheme in the same step
cudaError_t launch_births(bool fp64, const WsPtrs &W, const void *pools, int par, int max_blocks,
                          cudaStream_t s, int salt = 0);
// the sequential gas scheme, part 0 (channels below (13)) or 1 (above (14))
constexpr int DSMC_THREADS = 256;
cudaError_t launch_dsmc(bool fp64, const WsPtrs &W, const void *pools, int par, int part, cudaStream_t st);
// tile table of the current particle counts (after a sort), for the
// sequential scheme and its birth append
cudaError_t launch_retile(const WsPtrs &W, int par, cudaStream_t st);

// charge density -> Poisson -> field; per-step bookkeeping (mode 0), or a
// read-only evaluation of the fields of the current state (mode 1)
cudaError_t launch_field(bool fp64, bool diag, int mode, const WsPtrs &W, int par,
                         const LaunchCfg &L, cudaStream_t s);

cudaError_t launch_sort(bool fp64, const WsPtrs &W, const void *pools,
                        const int *sort_block_ds, const LaunchCfg &L, cudaStream_t s);
// Coulomb pass: a block per (cell, species) of COUL_THREADS threads; cells of
// at most COUL_STAGE particles are staged in shared memory
#ifndef O2_COUL_THREADS
#define O2_COUL_THREADS 384
#endif
#ifndef O2_COUL_STAGE
#define O2_COUL_STAGE 8192
#endif
constexpr int COUL_THREADS = O2_COUL_THREADS;
constexpr int COUL_STAGE = O2_COUL_STAGE;
size_t coulomb_smem_bytes(bool fp64);
cudaError_t launch_coulomb(bool fp64, const WsPtrs &W, const void *pools, int par, cudaStream_t st);
// inter-species Coulomb collisions of one species pair (0 e-O-, 1 e-O2+, 2 O- - O2+)
cudaError_t launch_coulomb_inter(bool fp64, const WsPtrs &W, const void *pools, int par, int pair,
                                 cudaStream_t st);
cudaError_t launch_pair(bool fp64, const WsPtrs &W, const void *pools, int par,
                        const LaunchCfg &L, cudaStream_t s);
// one reaction of the particle-target pass (k = 0, 1, 2 for (13), (14),
// (19)), and the append of (19)'s births
cudaError_t launch_pair_reaction(bool fp64, const WsPtrs &W, const void *pools, int par, int k,
                                 cudaStream_t s);
cudaError_t launch_pair_append(bool fp64, const WsPtrs &W, const void *pools, const LaunchCfg &L,
                               cudaStream_t s);
cudaError_t launch_load(bool fp64, const WsPtrs &W, const void *pools, const long long *d_ninit,
                        const double *d_vt, int max_n, cudaStream_t s);
cudaError_t launch_deposit_all(bool fp64, const WsPtrs &W, const void *pools, int disc,
                               int max_n, cudaStream_t s);
cudaError_t configure_kernels(bool fp64, LaunchCfg &L);

// text returned by pic_last_error(NULL) for calls without a handle
void set_last_error(const char *msg);

int kernels_per_sort();
int kernels_per_pair();

} // namespace o2
