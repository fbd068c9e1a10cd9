#include "heap_internal.h"
const smmo::MethodEntry g_methods_nbody[] = {{"nbody.none", 0, nullptr}};
const int g_methods_nbody_n = 0;
