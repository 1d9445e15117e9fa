// Cluster plane passes (plane_cluster.cu): the x-y transforms of one z-plane by a thread-block
// cluster whose CTAs transpose the plane through distributed shared memory, for planes larger
// than one CTA's shared memory.  FP32 transforms and fields.
#pragma once
#include "internal.h"

namespace hom {

// Chooses the cluster shape for g (fills pc_*); false if no shape fits (the split passes run).
bool plane_cluster_setup(Geo& g);
cudaError_t launch_plane_fwd_cluster(const FwdArgs<float, float>& a, int nrhs, cudaStream_t s);
cudaError_t launch_plane_inv_cluster(const InvArgs<float, float>& a, int nrhs, cudaStream_t s);

}  // namespace hom
