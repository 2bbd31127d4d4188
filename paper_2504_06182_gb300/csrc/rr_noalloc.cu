// rr_noalloc.cu -- rr_plan_noalloc: the planner of rr_plan for callers that
// must not allocate device memory.
//
// Who needs it: a reconfiguration control loop runs between imaging the trap
// array and driving the tweezers, once per cycle, under a hard deadline;
// cudaMalloc/cudaFree may synchronise the device and take unbounded time, so
// such a loop (and a plug-in whose device memory is owned by another
// allocator) cannot call them. This entry point needs no context and
// allocates nothing: its workspace is the file-scope array below, which
// every GPU that loads the library holds until the process exits.
//
// The call reads the move count back into a host variable and synchronises
// the stream before it returns, so it is refused (RR_ERR_ARG, nothing
// enqueued) on a stream that is being captured.
#include <cstring>
#include "rr_internal.cuh"

namespace rrk {
__global__ void k_plan_setup(rr_instance *, JobWS *, int, int, Arena);
__global__ void k_transpose(rr_instance *, JobWS *, int);
__global__ void k_colstats(rr_instance *, JobWS *, int, int);
__global__ void k_pair(rr_instance *, JobWS *, int);
__global__ void k_emit_cols(rr_instance *, JobWS *, int);
__global__ void k_emit_recv(rr_instance *, JobWS *, int);
}  // namespace rrk

using namespace rrk;

// Layout: descriptor at 0, workspace table at 256, arena bump pointer at
// 1024, arena from 4096 to the end.
static __device__ __align__(256) unsigned char g_noalloc_scratch[RR_NOALLOC_SCRATCH_BYTES];

static constexpr size_t OFF_INST = 0, OFF_WS = 256, OFF_TOP = 1024, OFF_ARENA = 4096;
static_assert(sizeof(rr_instance) <= OFF_WS - OFF_INST, "descriptor slot");
static_assert(sizeof(JobWS) <= OFF_TOP - OFF_WS, "workspace table slot");

// The planning set-up's arena requests for the largest accepted grid (side
// RR_NOALLOC_MAX_SIDE, target = the whole grid), each rounded up to the
// arena's 256-byte granule as the device allocator does.
static constexpr size_t pad256(size_t b) { return (b + 255) & ~(size_t)255; }
static constexpr size_t noalloc_worst_case()
{
    constexpr size_t S = RR_NOALLOC_MAX_SIDE, W = (S + 31) / 32;
    return pad256(sizeof(uint32_t) * S * W) +        // bit columns
           pad256(sizeof(int16_t) * S * S) +         // atom rows
           pad256(sizeof(int16_t) * S * S) +         // band holes (h = m, full width)
           pad256(sizeof(ColInfo) * S) + pad256(sizeof(RecvInfo) * S) +
           pad256(sizeof(Event) * (S + 1)) + pad256(sizeof(int32_t) * (2 * S + 1));
}
static_assert(noalloc_worst_case() <= RR_NOALLOC_SCRATCH_BYTES - OFF_ARENA,
              "the fixed workspace must hold the largest accepted plan");

// Device address of the scratch array, looked up once per device (host
// code must not use the symbol itself: it names a host-side stand-in).
static constexpr int MAX_DEVICES = 64;
static unsigned char *g_scratch_addr[MAX_DEVICES];

static int scratch_for_current_device(unsigned char **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return RR_ERR_CUDA;
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return RR_ERR_CUDA;
        g_scratch_addr[dev] = (unsigned char *)p;
    }
    *out = g_scratch_addr[dev];
    return RR_OK;
}

extern "C" int rr_plan_noalloc(const void *d_grid, int layout, int m, int n, rr_rect rect, rr_move *d_moves,
                               int64_t cap, int64_t *n_moves, cudaStream_t stream)
{
    if (!d_grid || !n_moves || (layout != RR_U8 && layout != RR_BITS32) || m < 1 || n < 1 ||
        m > RR_NOALLOC_MAX_SIDE || n > RR_NOALLOC_MAX_SIDE || rect.r0 < 0 || rect.r0 >= rect.r1 || rect.r1 > m ||
        rect.c0 < 0 || rect.c0 >= rect.c1 || rect.c1 > n || cap < 0 || (cap > 0 && !d_moves))
        return RR_ERR_ARG;
    cudaStreamCaptureStatus cap_st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cap_st) != cudaSuccess) return RR_ERR_CUDA;
    if (cap_st != cudaStreamCaptureStatusNone) return RR_ERR_ARG;   // it synchronises: not capturable
    unsigned char *base = nullptr;
    int st = scratch_for_current_device(&base);
    if (st != RR_OK) return st;
    rr_instance *d_inst = (rr_instance *)(base + OFF_INST);
    JobWS *d_ws = (JobWS *)(base + OFF_WS);
    Arena A;
    A.base = (char *)(base + OFF_ARENA);
    A.size = RR_NOALLOC_SCRATCH_BYTES - OFF_ARENA;
    A.top = (unsigned long long *)(base + OFF_TOP);

    rr_instance h;
    memset(&h, 0, sizeof(h));
    h.grid = d_grid; h.layout = layout; h.m = m; h.n = n; h.rect = rect;
    h.moves = d_moves; h.cap_moves = cap;
    // the previous call's contents remain: reset the bump pointer and the descriptor
    if (cudaMemsetAsync(A.top, 0, sizeof(unsigned long long), stream) != cudaSuccess) return RR_ERR_CUDA;
    if (cudaMemcpyAsync(d_inst, &h, sizeof(h), cudaMemcpyHostToDevice, stream) != cudaSuccess) return RR_ERR_CUDA;

    const int side = m > n ? m : n;
    const int colBlocks = (side + 7) / 8;
    const int tiles = ((side + 31) / 32) * ((side + 31) / 32);
    const int trBlocks = (tiles + 7) / 8;
    k_plan_setup<<<1, 128, 0, stream>>>(d_inst, d_ws, 1, side, A);
    k_transpose<<<dim3(trBlocks, 1), 256, 0, stream>>>(d_inst, d_ws, 1);
    k_colstats<<<dim3(colBlocks, 1), 256, 0, stream>>>(d_inst, d_ws, 1, 0);
    k_pair<<<1, 32, (size_t)side * 30 + 64, stream>>>(d_inst, d_ws, 1);
    k_emit_cols<<<dim3(colBlocks, 1), 256, 0, stream>>>(d_inst, d_ws, 1);
    k_emit_recv<<<dim3(side, 1), 256, 0, stream>>>(d_inst, d_ws, 1);
    if (cudaGetLastError() != cudaSuccess) return RR_ERR_CUDA;
    if (cudaMemcpyAsync(&h, d_inst, sizeof(h), cudaMemcpyDeviceToHost, stream) != cudaSuccess) return RR_ERR_CUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return RR_ERR_CUDA;
    *n_moves = h.n_moves;
    return h.status;
}
