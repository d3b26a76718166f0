// Streaming-pass instantiations for A stored as float.
#include "internal.h"

#define ROWPASS_TA float
#define ROWPASS_SUFFIX(name) name##_f32
#include "rowpass_dispatch.inc"
