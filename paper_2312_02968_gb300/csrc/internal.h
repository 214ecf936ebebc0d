// internal.h -- symbols shared between the library's translation units (not
// part of the C ABI).
#pragma once

// Record the text returned by mond_pm_last_error(NULL) on this thread.
void mond_pm_set_create_error(const char* msg);
