// step_fast_c01.cu -- launch configurations 0 and 1 of the double-float step kernel
// (a translation unit of their own, so that the configurations compile in
// parallel).
#include "step_fast_impl.cuh"

namespace sl {

void launch_fast_df_c0(const FastArgs &a, bool stats, bool debug, cudaStream_t s)
{
    launch_fast_df_cfg<256, 4>(a, stats, debug, s);
}

void launch_fast_df_c1(const FastArgs &a, bool stats, bool debug, cudaStream_t s)
{
    launch_fast_df_cfg<256, 3>(a, stats, debug, s);
}

}  // namespace sl
