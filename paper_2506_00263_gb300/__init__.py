"""GB300-native event-based Monte Carlo neutron transport with thread-data remapping."""
