"""GB300-native hot path of non-zero noise extrapolation (arXiv 2501.13237).

libnne.so (csrc/, built by build.py) holds every kernel of the path; nne.py
is its ctypes binding and runner.py the brickwork schedule above it.
"""
