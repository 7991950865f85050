// apax_select.cu -- the stream decision of Sec. 6 for containers with the
// sum stream (version 2), ahead of a single-array encode or profile sweep.
//
// Block j is coded on the stream that packed block j - 1 into the fewest
// bits at code 0 (block 0: its own), chosen among S0-S2 and the sum stream
// S3.  Sizing S3 as well in the sweep kernels would raise their register
// count for every container; this pass writes the decisions of a block
// range to a byte array that the sweeps read instead.  One team of TS
// threads per block, 128 threads per CTA.
#include "apax_team.cuh"
#include "apax_kernels.h"

namespace apax {
namespace {

template <int DT, int TS>
__global__ void __launch_bounds__(128) k_best_streams(SelArgs a)
{
    using raw = typename DT_<DT>::raw;
    const int team = threadIdx.x / TS;
    const uint64_t jl = (uint64_t)blockIdx.x * (blockDim.x / TS) + (uint64_t)team;
    const bool live = jl < a.count;
    const uint64_t j = a.j0 + jl;
    // the block whose code-0 sizes decide block j (every lane of the team
    // takes part in the team exchanges, live or not)
    TBlock<DT> pv;
    open_team_block<DT, TS>(pv, reinterpret_cast<const raw *>(a.x), a.n, a.N, live ? a.nb : 0,
                            j == 0 ? 0 : j - 1, a.gp, 0, a.gsh);
    const int s = team_best_stream<DT, TS>(pv, true);
    if (live && tlane<TS>() == 0) a.sel[jl] = (uint8_t)s;
}

template <int DT>
cudaError_t launch_dt(SelArgs a, cudaStream_t s)
{
    const int gs = a.gsh ? 8 : 4;
    // teams of 8 up to 2048 samples (at most 64 groups of 4 a thread),
    // teams of 32 above
    const bool big = a.N > 2048;
    const int ts = big ? 32 : 8;
    a.gp = gs == 8 ? 2 * (int)((a.N / 8 + ts - 1) / ts) : (int)((a.N / 4 + ts - 1) / ts);
    const uint64_t per = 128 / ts;
    const uint64_t ctas = (a.count + per - 1) / per;
    if (!ctas) return cudaSuccess;
    if (big) k_best_streams<DT, 32><<<(unsigned)ctas, 128, 0, s>>>(a);
    else k_best_streams<DT, 8><<<(unsigned)ctas, 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_best_streams(const SelArgs &a, cudaStream_t s)
{
    switch (a.dtype) {
    case 1: return launch_dt<1>(a, s);
    case 2: return launch_dt<2>(a, s);
    case 3: return launch_dt<3>(a, s);
    case 4: return launch_dt<4>(a, s);
    default: return launch_dt<5>(a, s);
    }
}

}  // namespace apax
