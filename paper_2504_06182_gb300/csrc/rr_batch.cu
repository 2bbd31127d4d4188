// rr_batch.cu -- kernels of the batching routine (arXiv 2504.06182, Alg. 4
// with the local constraint set of Sec. IV): each runs one stage of
// rr_batch.cuh over the instance array.
#include "rr_batch.cuh"

namespace rrk {

__global__ void k_bsetup(rr_instance *inst, JobWS *wsv, int count, Arena A, int lookback)
{
    s_bsetup(hw_blk(), inst, wsv, count, A, lookback);
}

__global__ void __launch_bounds__(LB_THREADS) k_pairoff_lookback(rr_instance *inst, JobWS *wsv, int count, Arena A)
{
    s_pairoff_lookback(hw_blk(), inst, wsv, count, A);
}

__global__ void k_gcount(rr_instance *inst, JobWS *wsv, int count)
{
    s_gcount(hw_blk(), inst, wsv, count);
}

__global__ void k_gscan(rr_instance *inst, JobWS *wsv, int count)
{
    s_gscan(hw_blk(), inst, wsv, count);
}

__global__ void k_gfill(rr_instance *inst, JobWS *wsv, int count)
{
    s_gfill(hw_blk(), inst, wsv, count);
}

__global__ void k_gsort(rr_instance *inst, JobWS *wsv, int count, int bufLen)
{
    s_gsort(hw_blk(), inst, wsv, count, bufLen);
}

__global__ void k_gsweep_h(rr_instance *inst, JobWS *wsv, int count, int lineCap)
{
    s_gsweep_h(hw_blk(), inst, wsv, count, lineCap);
}

__global__ void k_gsweep_v(rr_instance *inst, JobWS *wsv, int count, int lineCap)
{
    s_gsweep_v(hw_blk(), inst, wsv, count, lineCap);
}

__global__ void k_bsucc(rr_instance *inst, JobWS *wsv, int count)
{
    s_bsucc(hw_blk(), inst, wsv, count);
}

__global__ void k_brec(rr_instance *inst, JobWS *wsv, int count)
{
    s_brec(hw_blk(), inst, wsv, count);
}

__global__ void k_order(const rr_instance *inst, int count, int *perm)
{
    s_order(hw_blk(), inst, count, perm);
}

__global__ void k_gather(const rr_instance *inst, const int *perm, rr_instance *pinst)
{
    s_gather(hw_blk(), inst, perm, pinst);
}

__global__ void k_scatter(rr_instance *inst, const int *perm, const rr_instance *pinst, int count)
{
    s_scatter(hw_blk(), inst, perm, pinst, count);
}

__global__ void k_classify(rr_instance *inst, int count, int nclass, int max_side, int *classCount,
                           int *classList)
{
    s_classify(hw_blk(), inst, count, nclass, max_side, classCount, classList);
}

// 16-bit slot links (sides up to 256) and 32-bit ones; narrow (shared-memory
// slots only) and wide (overflow slots in global memory, for the instances
// the narrow pass handed over).
__global__ void k_sim16(rr_instance *inst, JobWS *wsv, int count, const int *classList, const int *classCount,
                        int slotCap, int lineCap)
{
    sim_body<int16_t, false>(hw_blk(), inst, wsv, count, classList, classCount, slotCap, lineCap);
}

__global__ void k_sim32(rr_instance *inst, JobWS *wsv, int count, const int *classList, const int *classCount,
                        int slotCap, int lineCap)
{
    sim_body<int32_t, false>(hw_blk(), inst, wsv, count, classList, classCount, slotCap, lineCap);
}

__global__ void k_sim16w(rr_instance *inst, JobWS *wsv, int count, const int *classList, const int *classCount,
                         int slotCap, int lineCap)
{
    sim_body<int16_t, true>(hw_blk(), inst, wsv, count, classList, classCount, slotCap, lineCap);
}

__global__ void k_sim32w(rr_instance *inst, JobWS *wsv, int count, const int *classList, const int *classCount,
                         int slotCap, int lineCap)
{
    sim_body<int32_t, true>(hw_blk(), inst, wsv, count, classList, classCount, slotCap, lineCap);
}

int guard_cap_batch(long long cap)
{
    return cudaMemcpyToSymbol(g_guard_cap, &cap, sizeof(cap)) == cudaSuccess ? RR_OK : RR_ERR_CUDA;
}

} // namespace rrk
