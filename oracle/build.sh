#!/bin/sh
# Builds the oracle shared library (test infrastructure only).
set -e
cd "$(dirname "$0")"
gcc -std=c11 -O2 -fno-fast-math -ffp-contract=off -fPIC -shared -Wall -Wextra -Wno-unused-parameter \
    -D_DEFAULT_SOURCE or_quad.c or_besser.c or_sweep.c or_see.c -lm -o liboracle.so
