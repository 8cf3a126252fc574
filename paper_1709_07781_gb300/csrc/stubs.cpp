// Entry points declared in ka.h whose implementation is not in this build yet.
#include "../../include/ka.h"

extern "C" {

ka_status ka_serve_run(ka_system *, const ka_serve_request *, uint32_t, const ka_serve_options *, ka_serve_result *,
                       ka_serve_stats *) {
    return KA_E_UNSUPPORTED;
}

}  // extern "C"
