"""B300-native engine for the plastic multi-compartment time-step loop of Plastic Arbor."""
