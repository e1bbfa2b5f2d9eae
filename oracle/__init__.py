"""CPU oracle of the forward Monte Carlo X-ray ray tracer.

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
benchmark's CPU-baseline leg may use it; the product path never does.
"""
