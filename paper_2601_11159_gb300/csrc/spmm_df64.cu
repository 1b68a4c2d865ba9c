// Double-float instantiations of the SpMM step (vectors as FP32 pairs, FP64 cross-thread sums).
#include "spmm.cuh"

namespace rd {

#define RD_DF64_ROWS(X) \
    X(2, 4) \
    X(2, 8) \
    X(2, 16) \
    X(2, 32) \
    X(4, 32) \
    X(1, 1)

#define RD_DF64_CONFIGS(X) \
    X(1, 1, 4)            \
    X(1, 1, 8)            \
    X(1, 1, 16)           \
    X(1, 1, 32)           \
    X(2, 4, 8)            \
    X(2, 8, 4)            \
    X(2, 16, 2)           \
    X(2, 4, 1)            \
    X(2, 8, 1)            \
    X(2, 16, 1)           \
    X(2, 32, 1)           \
    X(4, 32, 1)

// async row-stream (kind 3): two 8-byte elements per 16-byte lane slot, slabs of 16 to 64 columns
#define RD_DF64_ASYNC(X) \
    X(8)                \
    X(16)               \
    X(32)

bool launch_spmm_df64(const SpmmCfg& c, bool weighted, bool heavy, int grid, cudaStream_t st,
                     const StepArgs<df64>& a)
{
    if (c.kind == 3) {
        if (c.vec != 2 || c.nzl != 1) return false;
#define X(G) \
    if (c.gs == G) return launch_async_cfg<df64, G>(weighted, heavy, grid, st, a);
        RD_DF64_ASYNC(X)
#undef X
        return false;
    }
    if (c.kind == 2 && !heavy) return launch_spmv_tasks<df64>(weighted, grid, st, a);
    if (c.kind == 1 && !heavy) {
#define X(V, G) \
    if (c.vec == V && c.gs == G && c.nzl == 1) return launch_rows_cfg<df64, V, G>(weighted, grid, st, a);
        RD_DF64_ROWS(X)
#undef X
        return false;
    }
    // the heavy-row pre-pass runs the row-group heavy kernel with the same column tile and
    // one warp per chunk (heavy_cfg)
    const int zl = heavy ? heavy_cfg(c).nzl : c.nzl;
#define X(V, G, Z) \
    if (c.vec == V && c.gs == G && zl == Z) return launch_cfg<df64, V, G, Z>(weighted, heavy, grid, st, a);
    RD_DF64_CONFIGS(X)
#undef X
    return false;
}

int spmm_blocks_per_sm_df64(const SpmmCfg& c, bool weighted, bool heavy)
{
    if (c.kind == 3) {
        if (c.vec != 2 || c.nzl != 1) return 0;
#define X(G) \
    if (c.gs == G) return occupancy_async_cfg<df64, G>(weighted, heavy);
        RD_DF64_ASYNC(X)
#undef X
        return 0;
    }
    if (c.kind == 2 && !heavy) return occupancy_spmv_tasks<df64>(weighted);
    if (c.kind == 1 && !heavy) {
#define X(V, G) \
    if (c.vec == V && c.gs == G && c.nzl == 1) return occupancy_rows_cfg<df64, V, G>(weighted);
        RD_DF64_ROWS(X)
#undef X
        return 0;
    }
    const int zl = heavy ? heavy_cfg(c).nzl : c.nzl;
#define X(V, G, Z) \
    if (c.vec == V && c.gs == G && zl == Z) return occupancy_cfg<df64, V, G, Z>(weighted, heavy);
    RD_DF64_CONFIGS(X)
#undef X
    return 0;
}

std::vector<SpmmCfg> spmm_configs_df64()
{
    std::vector<SpmmCfg> v;
#define X(V, G, Z) v.push_back(SpmmCfg{V, G, Z, 0});
    RD_DF64_CONFIGS(X)
#undef X
    v.push_back(SpmmCfg{1, 1, 1, 2});
#define X(V, G) v.push_back(SpmmCfg{V, G, 1, 1});
    RD_DF64_ROWS(X)
#undef X
#define X(G) v.push_back(SpmmCfg{2, G, 1, 3});
    RD_DF64_ASYNC(X)
#undef X
    return v;
}

}  // namespace rd
