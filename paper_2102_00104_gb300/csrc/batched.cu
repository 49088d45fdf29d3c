// batched.cu -- batched and serve forms (many independent TT-SVDs).
#include "engine.h"
#include "tt_svd.h"

extern "C" {

tt_status tt_batched_query(int batch, const tt_job* jobs, size_t* work_bytes) {
  if (batch < 0 || (batch > 0 && !jobs) || !work_bytes) return TT_EINVAL;
  return TT_ENOTIMPL;
}

tt_status tt_svd_batched(int batch, const tt_job* jobs, void* work, size_t work_bytes,
                         void* stream) {
  (void)work; (void)work_bytes; (void)stream;
  if (batch < 0 || (batch > 0 && !jobs)) return TT_EINVAL;
  return TT_ENOTIMPL;
}

tt_status tt_serve_create(size_t hbm_budget_bytes, const tt_serve_opts* opts, tt_server** out) {
  (void)hbm_budget_bytes; (void)opts;
  if (!out) return TT_EINVAL;
  *out = nullptr;
  return TT_ENOTIMPL;
}
tt_status tt_serve_submit(tt_server* s, const tt_job* job, uint64_t* ticket) {
  (void)s; (void)job; (void)ticket;
  return TT_ENOTIMPL;
}
tt_status tt_serve_poll(tt_server* s, uint64_t ticket, int wait, tt_job_result* out) {
  (void)s; (void)ticket; (void)wait; (void)out;
  return TT_ENOTIMPL;
}
tt_status tt_serve_destroy(tt_server* s) {
  (void)s;
  return TT_ENOTIMPL;
}

}  // extern "C"
