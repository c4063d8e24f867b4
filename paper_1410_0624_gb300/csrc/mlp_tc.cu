// The learned form of cd_column_density in BF16 on the tcgen05 tensor cores.
#include "learned.cuh"

namespace cd {

cd_status column_density_learned_tc(cd_tree, cd_geom, const cd_opts &, float *, float *, float *, cudaStream_t)
{
    set_error("the BF16 learned form is not built yet");
    return CD_EUNSUPPORTED;
}

void net_free_tc(cd_net net)
{
    if (net->tc) cudaFree(net->tc);
    net->tc = nullptr;
}

}  // namespace cd
