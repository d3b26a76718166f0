// Streaming-pass instantiations for A stored as double.
#include "internal.h"

#define ROWPASS_TA double
#define ROWPASS_SUFFIX(name) name##_f64
#include "rowpass_dispatch.inc"
