// Library-internal entry of the batched form used by the served form.
#pragma once

#include "../../include/selm_mg.h"

namespace selm {

// A batch over existing handles (SELM_PROJ_NONE systems).  The handles are
// switched to their per-system coarse engines (no cooperative launches) and
// belong to the batch when `owns` is true; otherwise they outlive it and the
// caller destroys them after selm_batch_destroy.
selm_status batch_adopt(int nsys, selm_mg* const* hs, bool owns, void* stream, selm_batch** out);

}  // namespace selm
