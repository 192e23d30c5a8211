// placeholder, replaced by the tcgen05 kernel
#include "laph_internal.cuh"
namespace laph {
int tc_smem_bytes() { return 0; }
cudaError_t launch_tc(const InstDev *, const TileDev *, long long, const unsigned *, unsigned long long *,
                      const TcConfig &, int *, cudaStream_t)
{
    return cudaErrorNotSupported;
}
}  // namespace laph
