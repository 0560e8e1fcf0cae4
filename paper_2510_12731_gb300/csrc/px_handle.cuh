// Read access to a px_handle for library code outside px_api.cu.
#pragma once
#include <string>

#include "px.h"
#include "px_internal.cuh"

// The loaded structure, or nullptr when none is loaded.
const px::DevStructure* px_structure(const px_handle* h);
// The handle's own stream.
cudaStream_t px_stream(const px_handle* h);
// n and tau of Eq. 6 of the loaded structure.
double px_drude_n(const px_handle* h);
double px_tau(const px_handle* h);
// Store the message returned by px_last_error(h).
void px_set_error(px_handle* h, const std::string& msg);
