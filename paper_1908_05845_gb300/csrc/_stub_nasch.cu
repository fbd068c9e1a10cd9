#include "heap_internal.h"
const smmo::MethodEntry g_methods_nasch[] = {{"nasch.none", 0, nullptr}};
const int g_methods_nasch_n = 0;
