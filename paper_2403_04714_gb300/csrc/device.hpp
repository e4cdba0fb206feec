// device.hpp -- device views for host code (see abi_device.h).
#pragma once
#include "abi_device.h"
#include "compiler.hpp"
