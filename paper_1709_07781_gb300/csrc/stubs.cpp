// Entry points declared in ka.h whose implementation is not in this build yet.
#include "../../include/ka.h"

extern "C" {

ka_status ka_system_create(const ka_config *, ka_system **) { return KA_E_UNSUPPORTED; }
ka_status ka_system_destroy(ka_system *, int32_t) { return KA_E_UNSUPPORTED; }
ka_status ka_system_pool_bytes(ka_system *, uint64_t *, uint64_t *) { return KA_E_UNSUPPORTED; }
ka_status ka_ref_wrap(ka_system *, void *, uint64_t, uint64_t, ka_dtype, ka_access, ka_ref **) {
    return KA_E_UNSUPPORTED;
}
ka_status ka_ref_alloc(ka_system *, uint64_t, ka_dtype, ka_ref **) { return KA_E_UNSUPPORTED; }
ka_status ka_ref_count(ka_ref *, uint64_t *) { return KA_E_UNSUPPORTED; }
ka_status ka_ref_info(ka_ref *, void **, uint64_t *, int32_t *, int32_t *) { return KA_E_UNSUPPORTED; }
ka_status ka_ref_retain(ka_ref *) { return KA_E_UNSUPPORTED; }
ka_status ka_ref_release(ka_ref *) { return KA_E_UNSUPPORTED; }
ka_status ka_ref_serialize(const ka_ref *, void *, uint64_t, uint64_t *) { return KA_E_NOT_SERIALIZABLE; }
ka_status ka_spawn_stage(ka_system *, const ka_stage_desc *, ka_actor **) { return KA_E_UNSUPPORTED; }
ka_status ka_compose(ka_actor *, ka_actor *, ka_actor **) { return KA_E_UNSUPPORTED; }
ka_status ka_actor_arity(ka_actor *, int32_t *, int32_t *) { return KA_E_UNSUPPORTED; }
ka_status ka_actor_release(ka_actor *) { return KA_E_UNSUPPORTED; }
ka_status ka_request(ka_actor *, const ka_msg *, ka_request_h **) { return KA_E_UNSUPPORTED; }
ka_status ka_receive(ka_request_h *, int64_t, ka_msg *) { return KA_E_UNSUPPORTED; }
ka_status ka_debug_fail_stage(ka_actor *, int32_t) { return KA_E_UNSUPPORTED; }
ka_status ka_debug_kill_dispatcher(ka_system *) { return KA_E_UNSUPPORTED; }
ka_status ka_system_monitor(ka_system *, ka_monitor_fn, void *) { return KA_E_UNSUPPORTED; }
ka_status ka_actor_enable_graph(ka_actor *, int32_t) { return KA_E_UNSUPPORTED; }
ka_status ka_serve_run(ka_system *, const ka_serve_request *, uint32_t, const ka_serve_options *, ka_serve_result *,
                       ka_serve_stats *) {
    return KA_E_UNSUPPORTED;
}

}  // extern "C"
