// Host-side entry points of the CAPT library (builder, flattening, filters): internal,
// not part of the C ABI.  Kept apart from capt_internal.h, which holds the data layouts
// the kernels are compiled against.
#pragma once

#include "capt_internal.h"

namespace capt {

int build_host_tree(const float* points, size_t n, float r_min, float r_max, int threads, HostTree& out,
                    std::string& err);
void flatten(const HostTree& t, Layout& out);
int host_sfc_filter(const float* points, size_t n, float r, uint32_t* kept, size_t* n_out, std::string& err);
int host_morton_order(const float* points, size_t n, uint32_t* order, std::string& err);

}  // namespace capt
