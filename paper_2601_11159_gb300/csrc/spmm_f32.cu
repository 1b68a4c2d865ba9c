// FP32-vector instantiations of the SpMM step (FP32 vectors, FP64 cross-thread sums).
#include "spmm.cuh"

namespace rd {

#define RD_F32_CONFIGS(X) \
    X(1, 1, 4)            \
    X(1, 1, 8)            \
    X(1, 1, 16)           \
    X(1, 1, 32)           \
    X(4, 4, 1)            \
    X(4, 4, 2)            \
    X(4, 8, 1)            \
    X(4, 8, 2)            \
    X(4, 16, 1)           \
    X(4, 16, 2)           \
    X(4, 32, 1)           \
    X(8, 32, 1)

bool launch_spmm_f32(const SpmmCfg& c, bool weighted, bool heavy, int grid, cudaStream_t st,
                     const StepArgs<float>& a)
{
#define X(V, G, Z) \
    if (c.vec == V && c.gs == G && c.nzl == Z) return launch_cfg<float, V, G, Z>(weighted, heavy, grid, st, a);
    RD_F32_CONFIGS(X)
#undef X
    return false;
}

int spmm_blocks_per_sm_f32(const SpmmCfg& c, bool weighted, bool heavy)
{
#define X(V, G, Z) \
    if (c.vec == V && c.gs == G && c.nzl == Z) return occupancy_cfg<float, V, G, Z>(weighted, heavy);
    RD_F32_CONFIGS(X)
#undef X
    return 0;
}

std::vector<SpmmCfg> spmm_configs_f32()
{
    std::vector<SpmmCfg> v;
#define X(V, G, Z) v.push_back(SpmmCfg{V, G, Z});
    RD_F32_CONFIGS(X)
#undef X
    return v;
}

}  // namespace rd
