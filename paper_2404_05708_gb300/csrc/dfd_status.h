// dfd_status.h -- status codes shared by device and host code (from dfd.h).
#pragma once
#include "dfd.h"
