// Continuous-batching request loop (ccm_submit / ccm_poll).
#include "ccm_host.h"

namespace ccm {

struct Serving {};

void Context::shutdown_serving() {
  delete serving;
  serving = nullptr;
}

}  // namespace ccm
