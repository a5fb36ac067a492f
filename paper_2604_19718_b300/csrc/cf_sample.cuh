#pragma once
#include "cf_common.cuh"
