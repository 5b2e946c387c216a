// Internal declarations shared by the host builder and the CUDA translation
// unit of the mmpc library.
#pragma once

#include <cstddef>
#include <string>

#include "../../include/mmpc.h"

namespace mmpc {

// Offsets (in doubles) of the sections of the FP64 problem buffer; the order
// is the one documented at mmpc_build in mmpc.h.
struct ProblemLayout {
    size_t t, P, Pd, Pdd, lin, Q, K11x, K11y, K11p, K12p, K12x, K12y, C0x, C0y, C0p, total;
};

bool sizes_ok(int N, int n);
ProblemLayout layout(int N, int n);
std::string check_params(const mmpc_params* p);
void set_global_error(const std::string& msg);

}  // namespace mmpc
