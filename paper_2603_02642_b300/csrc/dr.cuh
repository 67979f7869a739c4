// NRTO-DR persistent kernel (Sec. III, Supplementary Sec. II).
#pragma once
#include "fulladmm.cuh"
