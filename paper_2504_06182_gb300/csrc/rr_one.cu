// rr_one.cu -- one grid planned and batched by ONE kernel launch.
//
// The paper's GPU red-rec (Sec. III.D, "single kernel implementation") runs
// the whole planner in one launch to keep the latency of one reconfiguration
// cycle low. Here one block of ONE_THREADS threads runs every stage of the
// multi-kernel path in turn -- planning (Alg. 1, or bird, Alg. 2), the
// conflict graph Gamma and the batching routine (Alg. 4) -- with a block
// barrier between stages instead of a kernel boundary. The stages are the
// same functions the separate kernels run (rr_plan.cuh, rr_bird.cuh,
// rr_batch.cuh), given block coordinates x = 0, gx = 1 so that each
// grid-stride loop covers all of its work with this block's warps; the
// single-warp stages (pairing, simulation) run on warp 0 and the two-warp
// bird stage on warps 0-1 while the other warps wait at the next barrier.
// The simulation keeps the ready set in registers (sim_small) while it stays
// within SMALL_CAP moves and falls back to the general one otherwise.
// The descriptor comes in as a kernel parameter and the final one is written
// to mapped host memory, so a call is one launch and one synchronisation.
#include <algorithm>
#include "rr_plan.cuh"
#include "rr_bird.cuh"
#include "rr_batch.cuh"

namespace rrk {

__global__ void __launch_bounds__(ONE_THREADS) k_one(rr_instance h, rr_instance *I, JobWS *ws, Arena A, int flags,
                                                      int side, int P2, rr_instance *hostOut)
{
    extern __shared__ int4 one_smem[];
    const Blk B{0, 0, 1};
    const int wid = threadIdx.x >> 5;
    const bool bird = (flags & RR_BIRD) != 0, batch = (flags & RR_WITH_BATCH) != 0;
    if (threadIdx.x == 0) {
        *I = h;
        *A.top = 0;
    }
    __syncthreads();
    s_plan_setup(B, I, ws, 1, side, A);
    __syncthreads();
    s_transpose(B, I, ws, 1);
    __syncthreads();
    s_colstats(B, I, ws, 1, (flags & RR_STRICT_RESERVOIR) ? 1 : 0);
    __syncthreads();
    if (bird) {
        if (wid < 2) s_bird(B, I, ws, 1, side);
        __syncthreads();
        s_emit_cols(B, I, ws, 1);
    } else {
        if (wid == 0) s_pair(B, I, ws, 1);
        __syncthreads();
        s_emit_cols(B, I, ws, 1);
        __syncthreads();
        s_emit_recv(B, I, ws, 1);
    }
    __syncthreads();
    if (batch && I->status == RR_OK) {          // read after a barrier: the same in every thread
        s_bsetup(B, I, ws, 1, A, 0);
        __syncthreads();
        s_gcount(B, I, ws, 1);
        __syncthreads();
        s_gscan(B, I, ws, 1);
        __syncthreads();
        s_gfill(B, I, ws, 1);
        __syncthreads();
        s_gsort(B, I, ws, 1, P2);
        __syncthreads();
        s_gsweep_h(B, I, ws, 1, side);
        __syncthreads();
        s_gsweep_v(B, I, ws, 1, side);
        __syncthreads();
        s_bsucc(B, I, ws, 1);
        __syncthreads();
        s_brec(B, I, ws, 1);
        __syncthreads();
        // the ready set in registers when it stays small; else the general
        // simulation (narrow pass, then the wide one if that runs out of slots)
        if (wid == 0) sim_small(I, ws[0], (char *)one_smem);
        __syncthreads();
        const bool general = I->status == RR_SIM_RETRY;
        __syncthreads();
        if (general) {
            if (threadIdx.x == 0) I->status = RR_OK;
            __syncthreads();
            const int slotCap = 2 * side + 8, lineCap = side;
            if (wid == 0) sim_body<int16_t, false>(B, I, ws, 1, nullptr, nullptr, slotCap, lineCap);
            __syncthreads();
            if (wid == 0) sim_body<int16_t, true>(B, I, ws, 1, nullptr, nullptr, slotCap, lineCap);
            __syncthreads();
        }
    }
    if (threadIdx.x < sizeof(rr_instance) / 4) ((volatile int32_t *)hostOut)[threadIdx.x] = ((int32_t *)I)[threadIdx.x];
}

// Dynamic shared memory of k_one for grids up to `side`: the largest
// request of its stages (pairing, bird, the Gamma sorts and sweeps with
// ONE_THREADS / 32 warps, the simulation).
size_t one_smem_bytes(int side, int flags)
{
    int P2 = 32;
    while (P2 < side) P2 <<= 1;
    const size_t warps = ONE_THREADS / 32;
    size_t b = (size_t)side * 30 + 64;                                       // pairing
    if (flags & RR_BIRD) {
        size_t cap = 1;
        while (cap < (size_t)side) cap <<= 1;
        b = std::max(b, 4 * ((size_t)side * ((side + 31) / 32) + 2 * cap) + 2 * 5 * (size_t)side);
    }
    if (flags & RR_WITH_BATCH) {
        b = std::max(b, warps * 4 * (size_t)P2);                              // k_gsort
        b = std::max(b, warps * 12 * (size_t)side);                           // k_gsweep_v (h needs a third)
        b = std::max(b, sim_smem_bytes(2 * side + 8, side, 2));
        b = std::max(b, small_smem_bytes());
    }
    return b;
}

const void *one_kernel() { return (const void *)k_one; }

int one_launch(rr_instance h, rr_instance *d_inst, JobWS *d_ws, Arena A, int flags, int side, size_t smem,
               rr_instance *hostOut, cudaStream_t s)
{
    int P2 = 32;
    while (P2 < side) P2 <<= 1;
    k_one<<<1, ONE_THREADS, smem, s>>>(h, d_inst, d_ws, A, flags, side, P2, hostOut);
    return cudaGetLastError() == cudaSuccess ? RR_OK : RR_ERR_CUDA;
}

int guard_cap_one(long long cap)
{
    return cudaMemcpyToSymbol(g_guard_cap, &cap, sizeof(cap)) == cudaSuccess ? RR_OK : RR_ERR_CUDA;
}

} // namespace rrk
