// rr_bird.cu -- kernel of the bird planner (arXiv 2504.06182, Alg. 2): the
// stage of rr_bird.cuh, one 64-thread block per instance.
#include "rr_bird.cuh"

namespace rrk {

__global__ void __launch_bounds__(64) k_bird(rr_instance *inst, JobWS *wsv, int count, int max_side)
{
    s_bird(hw_blk(), inst, wsv, count, max_side);
}

} // namespace rrk
