// rr_plan.cu -- kernels of the red-rec planner (arXiv 2504.06182, Alg. 1):
// each runs one stage of rr_plan.cuh over the instance array, blockIdx.y
// selecting the instance (blockIdx.x for the one-block-per-instance stages).
#include "rr_plan.cuh"

namespace rrk {

__global__ void k_plan_setup(rr_instance *inst, JobWS *wsv, int count, int max_side, Arena A)
{
    s_plan_setup(hw_blk(), inst, wsv, count, max_side, A);
}

__global__ void k_transpose(rr_instance *inst, JobWS *wsv, int count)
{
    s_transpose(hw_blk(), inst, wsv, count);
}

__global__ void k_colstats(rr_instance *inst, JobWS *wsv, int count, int strict)
{
    s_colstats(hw_blk(), inst, wsv, count, strict);
}

__global__ void k_pair(rr_instance *inst, JobWS *wsv, int count)
{
    s_pair(hw_blk(), inst, wsv, count);
}

__global__ void k_emit_cols(rr_instance *inst, JobWS *wsv, int count)
{
    s_emit_cols(hw_blk(), inst, wsv, count);
}

__global__ void k_emit_recv(rr_instance *inst, JobWS *wsv, int count)
{
    s_emit_recv(hw_blk(), inst, wsv, count);
}

int guard_cap_plan(long long cap)
{
    return cudaMemcpyToSymbol(g_guard_cap, &cap, sizeof(cap)) == cudaSuccess ? RR_OK : RR_ERR_CUDA;
}

} // namespace rrk
