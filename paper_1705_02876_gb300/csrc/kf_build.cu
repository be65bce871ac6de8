// Combinatorial track building (Sections 3 and 4.3).
#include "kf_api_internal.h"

namespace kf {

struct BuildState {
};

void destroy_build_state(BuildState *s) { delete s; }

}  // namespace kf
