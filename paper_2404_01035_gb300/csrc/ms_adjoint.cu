#include "ms_rt.h"
ms_status ms_before_step(ms_ctx*) { return MS_OK; }
void ms_reset_extra(ms_ctx*) {}
void ms_release_extra(ms_ctx*) {}
