// pd_net.h -- the warm-start network's device entry points used by the
// simulation (the public calls are in pd.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "pd.h"

namespace pd {

// Inference on B samples of H x W nodes on `stream`: sample b's nodes start
// at node index base[b] (device array) of x and y; the network's activation
// buffers use the same node indexing and must hold max(base) + H W nodes.
int net_forward_at(pd_net* net, const float* x, float* y, int B, int H, int W, const uint32_t* base,
                   int64_t node_span, cudaStream_t stream);
int64_t net_max_nodes(const pd_net* net);

}  // namespace pd
