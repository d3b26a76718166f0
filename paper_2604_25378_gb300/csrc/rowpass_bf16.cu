// Streaming-pass instantiations for A stored as __nv_bfloat16.
#include "internal.h"

#define ROWPASS_TA __nv_bfloat16
#define ROWPASS_SUFFIX(name) name##_bf16
#include "rowpass_dispatch.inc"
